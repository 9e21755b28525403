"""GPU parity of environment-map (emitter) derivatives vs the FP64 oracle.

PRB gradients w.r.t. the environment radiance, the forward-mode tangent along an
env direction, the radiance override (sampling keeps the scene's map), the
autograd wrapper and the wavefront variant.
"""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import GRAD_COSINE, PIXEL_FRACTION, cosine, rel_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi
    abi.load()
    return abi


def _scene():
    return S.spheres(n_spheres=6, level=2, grid=(3, 2), ground_quads=8, tex_res=256, width=64, height=48,
                     env_size=(64, 32))


def _settings(scene, **kw):
    from paper_2202_01284_gb300.render import RenderSettings
    cam = scene.cameras[0]
    base = dict(width=cam.width, height=cam.height, spp=8, max_depth=6, rr_depth=3, seed=5)
    base.update(kw)
    return RenderSettings(**base)


def _rin(oracle_mod, sc, st, env=None):
    return oracle_mod.render_in(sc.cameras[0], st.spp, st.max_depth, st.seed, st.rr_depth, st.nee,
                                crop=st.crop, env_radiance=env)


def _clean(ds, sc, st, oracle_mod):
    _, _, h = ds.forward(st, per_sample=True)
    _, _, refh = oracle_mod.render(oracle_mod.OracleScene(sc), _rin(oracle_mod, sc, st), per_sample=True)
    return (h[0].cpu().numpy().view(np.uint32) == refh.astype(np.uint32)).all(axis=-1)


def test_env_gradient_parity(lib, oracle_mod):
    from paper_2202_01284_gb300.render import DeviceScene
    sc = _scene()
    st = _settings(sc)
    ds = DeviceScene(sc, layout=1)
    osc = oracle_mod.OracleScene(sc)
    r = _rin(oracle_mod, sc, st)
    ref = oracle_mod.render(osc, r)
    T = oracle_mod.render(oracle_mod.OracleScene(sc.with_params(
        textures=[S.spheres_target_texture(sc.textures[0])])), r)
    gi = 2 * (ref - T) / ref.size + 1e-4  # a bias so that every pixel carries gradient
    _, _, _, ge_ref = oracle_mod.grad_tape(osc, r, gi, env=True)
    for nee in (True, False):
        st.nee = nee
        if not nee:
            r0 = _rin(oracle_mod, sc, st)
            _, _, _, ge_ref = oracle_mod.grad_tape(osc, r0, gi, env=True)
        ge = torch.zeros_like(ds.env)
        ds.backward(st, torch.as_tensor(gi[None], dtype=torch.float32, device="cuda"), g_env=ge)
        torch.cuda.synchronize()
        assert ds.status() == 0
        g = ge.cpu().numpy()
        c = cosine(g[..., :3], ge_ref[..., :3])
        rel = np.abs(g[..., :3] - ge_ref[..., :3]).max() / np.abs(ge_ref).max()
        print(f"nee={nee}: env grad cosine {c:.8f} max rel {rel:.2e}")
        assert c >= GRAD_COSINE
        assert rel < 1e-2
        assert not g[..., 3].any()


def test_env_override_and_jvp(lib, oracle_mod):
    from paper_2202_01284_gb300.render import DeviceScene
    sc = _scene()
    st = _settings(sc)
    ds = DeviceScene(sc, layout=1)
    base = ds.forward(st)
    same = ds.forward(st, env=ds.env.clone())
    rng = np.random.default_rng(4)
    env2 = sc.env.astype(np.float64) * rng.uniform(0.5, 2.0, size=sc.env.shape)
    img2 = ds.forward(st, env=torch.as_tensor(env2, dtype=torch.float32, device="cuda"))
    v = rng.random(sc.env.shape)
    v[..., 3] = 0
    img, dot = ds.jvp(st, t_env=torch.as_tensor(v, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(base, same)
    osc = oracle_mod.OracleScene(sc)
    ref2 = oracle_mod.render(osc, _rin(oracle_mod, sc, st, env=env2))
    _, ref_dot = oracle_mod.render_jvp(osc, _rin(oracle_mod, sc, st), t_env=v)
    clean = _clean(ds, sc, st, oracle_mod)
    ok2 = rel_ok(img2[0].cpu().numpy(), ref2).all(axis=-1)
    okd = rel_ok(dot[0].cpu().numpy(), ref_dot).all(axis=-1)
    print("clean", clean.mean(), "override ok", ok2[clean].mean(), "env jvp ok", okd[clean].mean())
    assert ok2.mean() >= PIXEL_FRACTION and okd.mean() >= PIXEL_FRACTION  # all pixels
    assert ok2[clean].mean() >= PIXEL_FRACTION
    assert okd[clean].mean() >= PIXEL_FRACTION


def test_env_autograd_and_wavefront(lib):
    import torch.autograd.forward_ad as fwAD
    from paper_2202_01284_gb300.render import DeviceScene, render
    sc = _scene()
    st = _settings(sc, seed=9)
    ds = DeviceScene(sc, layout=1)
    env = ds.env.clone().requires_grad_(True)
    img = render(ds, st, ds.albedo, ds.roughness, ds.textures, env=env)
    loss = (img ** 2).mean()
    loss.backward()
    gi = (2 * img.detach() / img.numel()).contiguous()
    g_ref = torch.zeros_like(ds.env)
    ds.backward(st, gi, g_env=g_ref)
    g_wf = torch.zeros_like(ds.env)
    ds.wavefront_backward(st, gi, g_env=g_wf)
    torch.cuda.synchronize()
    assert torch.allclose(env.grad, g_ref, rtol=1e-6, atol=0)
    assert cosine(g_wf.cpu().numpy(), g_ref.cpu().numpy()) >= 0.999999
    # forward AD through the wrapper = pt_render_jvp
    v = torch.rand_like(ds.env)
    with fwAD.dual_level():
        e = fwAD.make_dual(ds.env.clone(), v)
        out_t = fwAD.unpack_dual(render(ds, st, ds.albedo, ds.roughness, ds.textures, env=e)).tangent
    _, dot = ds.jvp(st, t_env=v)
    torch.cuda.synchronize()
    assert torch.equal(out_t, dot)


def test_env_arguments_rejected_without_env_map(lib):
    from paper_2202_01284_gb300.render import DeviceScene
    sc = S.cornell(width=16, height=16)
    ds = DeviceScene(sc)
    st = _settings(sc, spp=2, max_depth=3, rr_depth=-1)
    fake = torch.zeros((8, 16, 4), device="cuda")
    with pytest.raises(lib.PtError):
        ds.forward(st, env=fake)
    img = ds.forward(st)
    with pytest.raises(lib.PtError):
        ds.backward(st, torch.ones_like(img), g_env=fake)


def test_env_gradients_in_batched_launch(lib):
    """One persistent batch (forward + adjoint) with an env-gradient job equals the
    separate forward + backward launches with the same seeds."""
    from paper_2202_01284_gb300 import batch
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = _scene()
    ds = DeviceScene(sc, layout=1)
    cam = sc.cameras[0]
    target = torch.full((cam.height, cam.width, 3), 0.2, device="cuda")
    st = RenderSettings(width=cam.width, height=cam.height, spp=4, max_depth=8, rr_depth=3, seed=11,
                        lanes_per_pixel=4)
    img = ds.forward(st)[0]
    gi = (2 * (img - target) / img.numel())[None].contiguous()
    ge_ref = torch.zeros_like(ds.env)
    ds.backward(st, gi, g_env=ge_ref, seed=12)
    job = batch.Job(ds, cam, 4, seed=11, backward_seed=12, target=target, g_env=torch.zeros_like(ds.env))
    b = batch.Batch([job], tile=8, lanes_per_pixel=4, ctas_per_sm=2)
    b.run()
    torch.cuda.synchronize()
    assert torch.allclose(job.image, img, rtol=1e-5, atol=1e-7)
    c = cosine(job.g_env.cpu().numpy(), ge_ref.cpu().numpy())
    print("batched env grad cosine", c)
    assert c >= 0.999999
