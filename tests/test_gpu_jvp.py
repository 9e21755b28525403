"""GPU parity of the forward-mode image derivative (pt_render_jvp) vs the FP64 oracle.

A non-negative direction over albedo rows / texels makes every term of the
derivative non-negative, so image_dot is judged per pixel like the image
(1e-4 relative on 99.9 % of the pixels whose sample decisions agree with the
oracle's).  Signed directions (roughness) are judged by cosine, and the
JVP/VJP identity <gi, J v> = <J^T gi, v> ties pt_render_jvp to
pt_render_backward on the same seed.
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


def _settings(scene, **kw):
    from paper_2202_01284_gb300.render import RenderSettings
    cam = scene.cameras[0]
    base = dict(width=cam.width, height=cam.height, spp=4, max_depth=4, seed=7)
    base.update(kw)
    return RenderSettings(**base)


def _rin(oracle_mod, sc, st):
    return oracle_mod.render_in(sc.cameras[0], st.spp, st.max_depth, st.seed, st.rr_depth, st.nee, crop=st.crop)


def _clean_pixels(ds, sc, st, oracle_mod):
    """Pixels whose every sample takes the oracle's decisions (forward fingerprints)."""
    _, _, h = ds.forward(st, per_sample=True)
    _, _, refh = oracle_mod.render(oracle_mod.OracleScene(sc), _rin(oracle_mod, sc, st), per_sample=True)
    return (h[0].cpu().numpy().view(np.uint32) == refh.astype(np.uint32)).all(axis=-1)


def _t(x):
    return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("layout", [0, 1])
def test_cornell_albedo_jvp_parity(lib, oracle_mod, layout):
    from paper_2202_01284_gb300.render import DeviceScene
    sc = S.cornell()
    st = _settings(sc, spp=4, max_depth=5, seed=7)
    ds = DeviceScene(sc, layout=layout)
    rng = np.random.default_rng(1)
    v = rng.random(sc.albedo.shape)
    img, dot = ds.jvp(st, t_albedo=_t(v))
    fwd = ds.forward(st)
    torch.cuda.synchronize()
    assert ds.status() == 0
    img, dot, fwd = img[0].cpu().numpy(), dot[0].cpu().numpy(), fwd[0].cpu().numpy()
    ref_img, ref_dot = oracle_mod.render_jvp(oracle_mod.OracleScene(sc), _rin(oracle_mod, sc, st), t_albedo=v)
    clean = _clean_pixels(ds, sc, st, oracle_mod)
    ok_img = rel_ok(img, ref_img).all(axis=-1)
    ok_dot = rel_ok(dot, ref_dot).all(axis=-1)
    print("clean", clean.mean(), "img ok", ok_img[clean].mean(), "dot ok", ok_dot[clean].mean(),
          "all pixels: img", ok_img.mean(), "dot", ok_dot.mean(), "divergent", int((~clean).sum()), "of", clean.size)
    assert ok_img.mean() >= PIXEL_FRACTION and ok_dot.mean() >= PIXEL_FRACTION  # all pixels (measured 1.0)
    assert ok_img[clean].mean() >= PIXEL_FRACTION
    assert ok_dot[clean].mean() >= PIXEL_FRACTION
    # the primal of the JVP pass is the forward render
    assert rel_ok(img, fwd, rel=1e-5).all(axis=-1).mean() >= PIXEL_FRACTION


def test_cornell96_texel_and_roughness_jvp(lib, oracle_mod):
    from paper_2202_01284_gb300.render import DeviceScene
    sc = S.cornell96(width=512, height=512)
    crop = (192, 160, 96, 80)
    st = _settings(sc, spp=8, max_depth=6, seed=21, crop=crop)
    ds = DeviceScene(sc, layout=1)
    rng = np.random.default_rng(2)
    vt = rng.random(sc.textures[0].shape)
    vt[..., 3] = 0
    va = rng.random(sc.albedo.shape) if sc.albedo.size else None
    _, dot = ds.jvp(st, t_albedo=_t(va), t_textures=[_t(vt)])
    torch.cuda.synchronize()
    dot = dot[0].cpu().numpy()
    osc = oracle_mod.OracleScene(sc)
    r = _rin(oracle_mod, sc, st)
    _, ref_dot = oracle_mod.render_jvp(osc, r, t_albedo=va, t_textures=[vt])
    clean = _clean_pixels(ds, sc, st, oracle_mod)
    ok = rel_ok(dot, ref_dot).all(axis=-1)
    print("texel jvp: clean", clean.mean(), "ok", ok[clean].mean(), "all", ok.mean(),
          "divergent", int((~clean).sum()), "of", clean.size)
    # all pixels: measured 0.99557 (40 divergent of 7680: texel edges of the 2048^2 atlas at 8 spp x 6 vertices)
    assert ok.mean() >= 0.99 and (~clean).sum() <= 80
    assert ok[clean].mean() >= PIXEL_FRACTION
    # roughness: signed derivative, judged by cosine over the crop
    vr = rng.normal(size=sc.roughness.shape)
    _, dot_r = ds.jvp(st, t_roughness=_t(vr))
    torch.cuda.synchronize()
    _, ref_r = oracle_mod.render_jvp(osc, r, t_rough=vr)
    c = cosine(dot_r[0].cpu().numpy()[clean], ref_r[clean])
    print("roughness jvp cosine", c)
    assert c >= GRAD_COSINE


def test_spheres_jvp_parity(lib, oracle_mod):
    """GGX conductor, dielectric, textured diffuse, env map, roulette."""
    from paper_2202_01284_gb300.render import DeviceScene
    sc = S.spheres(n_spheres=6, level=2, grid=(3, 2), ground_quads=8, tex_res=256, width=64, height=48)
    st = _settings(sc, spp=8, max_depth=8, rr_depth=3, seed=5)
    ds = DeviceScene(sc, layout=1)
    rng = np.random.default_rng(3)
    vt = [rng.random(t.shape) for t in sc.textures]
    for t in vt:
        t[..., 3] = 0
    va = rng.random(sc.albedo.shape) if sc.albedo.size else None
    _, dot = ds.jvp(st, t_albedo=_t(va), t_textures=[_t(t) for t in vt])
    torch.cuda.synchronize()
    dot = dot[0].cpu().numpy()
    _, ref_dot = oracle_mod.render_jvp(oracle_mod.OracleScene(sc), _rin(oracle_mod, sc, st), t_albedo=va,
                                       t_textures=vt)
    clean = _clean_pixels(ds, sc, st, oracle_mod)
    ok = rel_ok(dot, ref_dot).all(axis=-1)
    print("spheres jvp: clean", clean.mean(), "ok", ok[clean].mean(), "all", ok.mean(),
          "divergent", int((~clean).sum()), "of", clean.size)
    assert ok.mean() >= PIXEL_FRACTION  # all pixels (measured 0.99967, 1 divergent of 3072)
    assert ok[clean].mean() >= PIXEL_FRACTION


def test_jvp_vjp_identity_on_gpu(lib):
    """<gi, jvp(v)> == <backward(gi), v> with the same seed: both passes replay the
    same paths, so this holds up to FP32 summation order."""
    from paper_2202_01284_gb300.render import DeviceScene
    sc = S.cornell96(width=96, height=96)
    st = _settings(sc, spp=4, max_depth=5, seed=13)
    ds = DeviceScene(sc, layout=1)
    g = torch.Generator(device="cuda").manual_seed(4)
    va = torch.randn(ds.albedo.shape, device="cuda", generator=g) if ds.albedo.numel() else None
    vt = torch.randn(ds.textures[0].shape, device="cuda", generator=g)
    vt[..., 3] = 0
    vr = torch.randn(ds.roughness.shape, device="cuda", generator=g)
    _, dot = ds.jvp(st, t_albedo=va, t_textures=[vt], t_roughness=vr)
    gi = torch.randn(dot.shape, device="cuda", generator=g)
    ga = torch.zeros_like(ds.albedo) if va is not None else None
    gt = torch.zeros_like(ds.textures[0])
    gr = torch.zeros_like(ds.roughness)
    ds.backward(st, gi, g_albedo=ga, g_textures=[gt], g_roughness=gr)
    torch.cuda.synchronize()
    lhs = float((gi.double() * dot.double()).sum())
    rhs = float((gt.double() * vt.double()).sum() + (gr.double() * vr.double()).sum())
    if ga is not None:
        rhs += float((ga.double() * va.double()).sum())
    print("jvp/vjp identity", lhs, rhs)
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))


def test_forward_ad_through_render_fn(lib):
    """torch.autograd.forward_ad on RenderFn gives pt_render_jvp's tangent."""
    import torch.autograd.forward_ad as fwAD
    from paper_2202_01284_gb300.render import DeviceScene, render
    sc = S.cornell(width=32, height=32)
    ds = DeviceScene(sc)
    st = _settings(sc, spp=4, max_depth=4, seed=5)
    v = torch.rand(ds.albedo.shape, device="cuda")
    with fwAD.dual_level():
        alb = fwAD.make_dual(ds.albedo.clone(), v)
        img = render(ds, st, alb, ds.roughness.clone(), [])
        out_t = fwAD.unpack_dual(img).tangent
    _, dot = ds.jvp(st, t_albedo=v)
    torch.cuda.synchronize()
    assert out_t is not None
    assert torch.equal(out_t, dot)


def test_jvp_bad_arguments(lib):
    from paper_2202_01284_gb300.render import DeviceScene
    sc = S.cornell96(width=32, height=32, tex_res=64)
    ds = DeviceScene(sc)
    st = _settings(sc)
    wrong = torch.zeros((8, 8, 4), device="cuda")
    with pytest.raises(lib.PtError) as e:
        ds.jvp(st, t_textures=[wrong])
    assert e.value.code == lib.PT_ERR_ARG
    if ds.albedo.shape[0] > 1:  # a direction with fewer albedo rows than the scene references
        with pytest.raises(lib.PtError):
            ds.jvp(st, t_albedo=torch.zeros((ds.albedo.shape[0] - 1, 3), device="cuda"))
    st.spp = 0
    with pytest.raises(lib.PtError):
        ds.jvp(st)
