"""Parity at the full throughput workload, in the launch configuration the bench times.

196,608-triangle sphere scene, 1024x1024, 64 spp, depth 8, roulette from 3, 8-wide
BVH, automatic launch shape -- the production (non-instrumented) forward and PRB
adjoint kernels over the whole image.  The FP64 oracle computes sampled 16x16
crops (sky, spheres, ground) one by one; the GPU's decision fingerprints of the
same crops (instrumented launch, same seeds) mark the pixels whose samples all
took the oracle's decisions, and those must meet the 1e-4 bar on 99.9 %.
Gradients: dLoss/dI is non-zero on the crops only, so the full-image adjoint and
the oracle's tape on the crops differentiate the same function.
"""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import GRAD_COSINE, PIXEL_FRACTION, cosine, rel_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CROPS = [(496, 40, 16, 16), (400, 540, 16, 16), (600, 600, 16, 16), (300, 720, 16, 16)]

# Path-divergence budget at this workload (64 samples of up to 8 vertices per pixel):
# measured 6 divergent pixels of 1024 (0.59 %), every one of them the only kind of
# pixel that misses 1e-4; all pixels together 0.9941.  The 0.1 % budget holds on the
# 36-triangle box (all pixels 1.0); here FP32-versus-FP64 decisions at triangle and
# texel edges flip about 1 path in 10^4, and a pixel of 64 such paths takes one
# flip with probability near 0.6 %.
MAX_DIVERGENT_PIXELS = 12
ALL_PIXEL_FRACTION = 0.99


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    abi.load()
    sc = S.spheres()
    ds = DeviceScene(sc, layout=abi.PT_BVH_WIDE)
    st = RenderSettings(width=1024, height=1024, spp=64, max_depth=8, rr_depth=3, seed=11)
    return sc, ds, st


def test_fullsize_forward_parity_on_crops(full, oracle_mod):
    from dataclasses import replace
    sc, ds, st = full
    img = ds.forward(st)[0].cpu().numpy()
    osc = oracle_mod.OracleScene(sc)
    clean_ok, clean_n, all_ok, all_n, divergent = 0, 0, 0, 0, 0
    for crop in CROPS:
        x0, y0, w, h = crop
        ref, _, refh = oracle_mod.render(osc, oracle_mod.render_in(sc.cameras[0], 64, 8, 11, 3, True, crop=crop),
                                         per_sample=True)
        _, _, gh = ds.forward(replace(st, crop=crop), per_sample=True)
        clean = (gh[0].cpu().numpy().view(np.uint32) == refh.astype(np.uint32)).all(axis=-1)
        ok = rel_ok(img[y0:y0 + h, x0:x0 + w], ref).all(axis=-1)
        print(crop, "clean", clean.mean(), "ok on clean", ok[clean].mean(), "ok all", ok.mean(),
              "divergent", int((~clean).sum()), "of", clean.size)
        clean_ok += int(ok[clean].sum())
        clean_n += int(clean.sum())
        all_ok += int(ok.sum())
        all_n += int(ok.size)
        divergent += int((~clean).sum())
    print(f"full-size forward: all pixels {all_ok / all_n:.5f}, clean pixels {clean_ok / clean_n:.5f}, "
          f"divergent pixels {divergent} of {all_n}")
    assert clean_ok / clean_n >= PIXEL_FRACTION
    assert divergent <= MAX_DIVERGENT_PIXELS
    assert all_ok / all_n >= ALL_PIXEL_FRACTION


def test_fullsize_adjoint_parity_on_crops(full, oracle_mod):
    sc, ds, st = full
    rng = np.random.default_rng(5)
    gi = np.zeros((1024, 1024, 3), np.float32)
    osc = oracle_mod.OracleScene(sc)
    gt_ref = np.zeros(sc.textures[0].shape)
    gr_ref = np.zeros(sc.roughness.shape)
    for crop in CROPS:
        x0, y0, w, h = crop
        g = rng.random((h, w, 3)).astype(np.float32) * 1e-3
        gi[y0:y0 + h, x0:x0 + w] = g
        _, gt, gr = oracle_mod.grad_tape(osc, oracle_mod.render_in(sc.cameras[0], 64, 8, 11, 3, True, crop=crop), g)
        gt_ref += gt[0]
        gr_ref += gr
    g_tex = torch.zeros_like(ds.textures[0])
    g_rough = torch.zeros_like(ds.roughness)
    ds.backward(st, torch.as_tensor(gi[None], device="cuda"), g_textures=[g_tex], g_roughness=g_rough)
    torch.cuda.synchronize()
    assert ds.status() == 0
    c_t = cosine(g_tex.cpu().numpy()[..., :3], gt_ref[..., :3])
    c_r = cosine(g_rough.cpu().numpy(), gr_ref)
    rel_r = np.abs(g_rough.cpu().numpy() - gr_ref).max() / np.abs(gr_ref).max()
    print(f"full-size adjoint: texture cosine {c_t:.7f}, roughness cosine {c_r:.9f} (max rel {rel_r:.2e})")
    assert c_r >= GRAD_COSINE
    assert c_t >= GRAD_COSINE  # measured 0.9999981
