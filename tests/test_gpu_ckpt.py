"""GPU parity of reverse mode with checkpoints (pt_ckpt_forward / pt_ckpt_backward).

The checkpointed reverse sweep computes the same estimator as PRB with the
forward's seed, so its gradients are held to the oracle's stored-tape gradients
(the oracle's tape is itself a checkpointed reverse mode) and to PRB on the GPU.
"""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import GRAD_COSINE, cosine

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
    base = dict(width=cam.width, height=cam.height, spp=8, max_depth=6, seed=21)
    base.update(kw)
    return RenderSettings(**base)


def test_ckpt_gradients_match_oracle_and_prb(lib, oracle_mod):
    from paper_2202_01284_gb300.render import Checkpoints, DeviceScene, ckpt_backward, ckpt_forward
    sc = S.cornell96(width=512, height=512)
    crop = (192, 160, 96, 96)
    st = _settings(sc, crop=crop)
    ds = DeviceScene(sc, layout=1)
    ck = Checkpoints(96 * 96 * 8, 6)
    assert ck.nbytes == 96 * 96 * 8 * (6 * 64 + 4)
    img = ckpt_forward(ds, st, ck)
    mega = ds.forward(st)
    torch.cuda.synchronize()
    assert torch.allclose(img, mega, rtol=1e-6, atol=0)
    r = oracle_mod.render_in(sc.cameras[0], st.spp, st.max_depth, st.seed, crop=crop)
    osc = oracle_mod.OracleScene(sc)
    ref = oracle_mod.render(osc, r)
    tgt = sc.with_params(textures=[S.cornell96_target_texture(sc.textures[0])])
    T = oracle_mod.render(oracle_mod.OracleScene(tgt), oracle_mod.render_in(sc.cameras[0], 8, 6, 23, crop=crop))
    gi = 2 * (ref - T) / ref.size
    _, gt_ref, gr_ref = oracle_mod.grad_tape(osc, r, gi)
    gi_t = torch.as_tensor(gi[None], dtype=torch.float32, device="cuda")
    gt, gr = torch.zeros_like(ds.textures[0]), torch.zeros_like(ds.roughness)
    ckpt_backward(ds, st, ck, gi_t, g_textures=[gt], g_roughness=gr)
    gt_p, gr_p = torch.zeros_like(ds.textures[0]), torch.zeros_like(ds.roughness)
    ds.backward(st, gi_t, g_textures=[gt_p], g_roughness=gr_p)
    torch.cuda.synchronize()
    assert ds.status() == 0
    c_t, c_r = cosine(gt.cpu().numpy()[..., :3], gt_ref[0][..., :3]), cosine(gr.cpu().numpy(), gr_ref)
    c_tp, c_rp = cosine(gt.cpu().numpy(), gt_p.cpu().numpy()), cosine(gr.cpu().numpy(), gr_p.cpu().numpy())
    print(f"ckpt vs oracle: tex {c_t:.7f} rough {c_r:.7f}; vs PRB: tex {c_tp:.9f} rough {c_rp:.9f}")
    assert c_r >= GRAD_COSINE and c_t >= GRAD_COSINE
    assert c_tp >= 0.99999 and c_rp >= 0.99999
    rel = (gr - gr_p).abs().max().item() / gr_p.abs().max().item()
    assert rel < 1e-3


def test_ckpt_env_gradients_and_roulette(lib, oracle_mod):
    from paper_2202_01284_gb300.render import Checkpoints, DeviceScene, ckpt_backward, ckpt_forward
    sc = S.spheres(n_spheres=6, level=2, grid=(3, 2), ground_quads=8, tex_res=256, width=64, height=48,
                   env_size=(64, 32))
    st = _settings(sc, spp=8, max_depth=8, rr_depth=3, seed=5)
    ds = DeviceScene(sc, layout=1)
    ck = Checkpoints(64 * 48 * 8, 8)
    img = ckpt_forward(ds, st, ck)
    r = oracle_mod.render_in(sc.cameras[0], 8, 8, 5, 3, True)
    osc = oracle_mod.OracleScene(sc)
    gi = np.full((48, 64, 3), 1e-3) + 1e-3 * np.random.default_rng(2).random((48, 64, 3))
    ga, gt_ref, gr_ref, ge_ref = oracle_mod.grad_tape(osc, r, gi, env=True)
    gi_t = torch.as_tensor(gi[None], dtype=torch.float32, device="cuda")
    ge, gt, gr = torch.zeros_like(ds.env), torch.zeros_like(ds.textures[0]), torch.zeros_like(ds.roughness)
    ckpt_backward(ds, st, ck, gi_t, g_textures=[gt], g_roughness=gr, g_env=ge)
    torch.cuda.synchronize()
    assert ds.status() == 0
    c_e = cosine(ge.cpu().numpy(), ge_ref)
    c_t = cosine(gt.cpu().numpy()[..., :3], gt_ref[0][..., :3])
    c_r = cosine(gr.cpu().numpy(), gr_ref)
    print(f"spheres ckpt vs oracle: env {c_e:.8f} tex {c_t:.7f} rough {c_r:.7f}")
    assert c_e >= GRAD_COSINE and c_r >= GRAD_COSINE and c_t >= GRAD_COSINE


def test_ckpt_capacity_checks(lib):
    from paper_2202_01284_gb300.render import Checkpoints, DeviceScene, ckpt_backward, ckpt_forward
    sc = S.cornell(width=16, height=16)
    ds = DeviceScene(sc)
    ck = Checkpoints(16 * 16 * 4, 4)
    st = _settings(sc, spp=4, max_depth=4)
    img = ckpt_forward(ds, st, ck)
    for bad in (dict(spp=5), dict(max_depth=5)):
        with pytest.raises(lib.PtError) as e:
            ckpt_forward(ds, _settings(sc, **{**dict(spp=4, max_depth=4), **bad}), ck)
        assert e.value.code == lib.PT_ERR_ARG
    # a backward with a shallower depth than the stored checkpoints stays in bounds
    g = torch.zeros_like(ds.albedo)
    ckpt_backward(ds, _settings(sc, spp=4, max_depth=2), ck, torch.ones_like(img), g_albedo=g)
    torch.cuda.synchronize()
    assert torch.isfinite(g).all()
