"""Persistent lane scheduling against one unit per thread (through the C ABI).

Both schedules trace the same samples from the same PCG32 streams; only the order in
which lanes take (pixel, lane) units differs.  With one lane per pixel the film is a
plain store and the images agree bit for bit; with several lanes per pixel the
persistent forward adds lane sums with float atomics, so images agree to FP32
rounding of a sum of at most 32 terms.  The replay's gradients are scattered with
atomics in both schedules (order-dependent rounding only), the split radiance pass
stores per-sample radiance (identical)."""
from dataclasses import replace

import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import cosine, pixel_ok_fraction, PIXEL_FRACTION

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi
    abi.load()
    return abi


def _scene(lib):
    from paper_2202_01284_gb300.render import DeviceScene
    sc = S.spheres(n_spheres=6, level=2, grid=(3, 2), ground_quads=8, tex_res=256, width=67, height=45)
    return sc, DeviceScene(sc, layout=lib.PT_BVH_WIDE)


def _st(**kw):
    from paper_2202_01284_gb300.render import RenderSettings
    base = dict(width=67, height=45, spp=12, max_depth=8, rr_depth=3, seed=9)
    base.update(kw)
    return RenderSettings(**base)


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 32])
def test_forward_persistent_equals_static(lib, lanes):
    sc, ds = _scene(lib)
    for crop in (None, (3, 5, 41, 29)):
        st = _st(lanes_per_pixel=lanes, crop=crop)
        a = ds.forward(replace(st, schedule=lib.PT_SCHED_PERSISTENT))
        b = ds.forward(replace(st, schedule=lib.PT_SCHED_STATIC))
        torch.cuda.synchronize()
        assert ds.status() == 0
        if lanes == 1:
            assert torch.equal(a, b), crop
        else:
            assert torch.allclose(a, b, rtol=2e-6, atol=1e-7), (crop, float((a - b).abs().max()))


def test_two_cameras_and_tiny_launches(lib):
    """Fewer units than one CTA holds; several cameras; a 1x1 crop."""
    sc, ds = _scene(lib)
    cams = [sc.cameras[0], S.Camera((1.0, 2.5, 7.0), (0.0, 0.4, 0.0), (0.0, 1.0, 0.0), 50.0, 67, 45)]
    for crop, lanes in (((10, 10, 1, 1), 4), ((0, 0, 5, 3), 8), (None, 8)):
        st = _st(lanes_per_pixel=lanes, crop=crop)
        a = ds.forward(replace(st, schedule=lib.PT_SCHED_PERSISTENT), cams=cams)
        b = ds.forward(replace(st, schedule=lib.PT_SCHED_STATIC), cams=cams)
        torch.cuda.synchronize()
        assert torch.allclose(a, b, rtol=2e-6, atol=1e-7), crop


def test_split_adjoint_and_forward_mode(lib):
    sc, ds = _scene(lib)
    st = _st(lanes_per_pixel=4)
    rng = np.random.default_rng(4)
    gi = torch.as_tensor(rng.random((1, 45, 67, 3)).astype(np.float32) * 1e-3, device="cuda")
    t = [torch.as_tensor(rng.random(x.shape).astype(np.float32), device="cuda") for x in ds.textures]
    out = []
    for sched in (lib.PT_SCHED_PERSISTENT, lib.PT_SCHED_STATIC):
        gt = torch.zeros_like(ds.textures[0])
        gr = torch.zeros_like(ds.roughness)
        ds.backward(replace(st, schedule=sched, prb_mode=lib.PT_PRB_SPLIT), gi, g_textures=[gt], g_roughness=gr,
                    seed=21)
        img, dot = ds.jvp(replace(st, schedule=sched), t_textures=t)
        torch.cuda.synchronize()
        assert ds.status() == 0
        out.append((gt.cpu().numpy(), gr.cpu().numpy(), img.cpu().numpy(), dot.cpu().numpy()))
    (gt0, gr0, i0, d0), (gt1, gr1, i1, d1) = out
    assert np.abs(gt1).sum() > 0 and np.abs(gr1).sum() > 0
    assert cosine(gt0, gt1) > 0.999999 and cosine(gr0, gr1) > 0.999999
    assert np.allclose(gr0, gr1, rtol=1e-4, atol=1e-9)
    assert pixel_ok_fraction(i0, i1, rel=1e-5)[0] >= PIXEL_FRACTION
    assert pixel_ok_fraction(d0, d1, rel=1e-5)[0] >= PIXEL_FRACTION


def test_schedule_argument_checked(lib):
    sc, ds = _scene(lib)
    with pytest.raises(lib.PtError):
        ds.forward(_st(schedule=3))
