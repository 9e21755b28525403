"""pt_render_batch_noalloc: the batched render for callers that may not allocate
device memory (for example a plugin whose host application owns the whole
device-memory budget).  Its scratch sits in a static device array; this test
checks, through the C ABI, that two calls in a row give the same images and
gradients as the allocating entry point pt_render_batch."""
import pytest

from paper_2202_01284_gb300 import scenes as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _setup():
    from paper_2202_01284_gb300 import abi, batch, render
    abi.load()
    a = S.spheres(n_spheres=4, level=2, grid=(2, 2), ground_quads=8, tex_res=64)
    b = S.spheres(5, n_spheres=3, level=3, grid=(3, 1), ground_quads=16, tex_res=128)
    scenes = [render.DeviceScene(a, layout=abi.PT_BVH_WIDE), render.DeviceScene(b, layout=abi.PT_BVH_WIDE)]
    cams = [(0, S.Camera((0.0, 3.0, 8.0), (0.0, 0.4, 0.0), (0.0, 1.0, 0.0), 45.0, 37, 53), 4),
            (1, S.Camera((1.0, 2.5, 7.0), (0.0, 0.4, 0.0), (0.0, 1.0, 0.0), 50.0, 64, 32), 8),
            (0, S.Camera((-2.0, 2.0, 6.0), (0.0, 0.4, 0.0), (0.0, 1.0, 0.0), 40.0, 20, 20), 2)]
    jobs = []
    for k, (si, cam, spp) in enumerate(cams):
        ds = scenes[si]
        jobs.append(batch.Job(ds, cam, spp, seed=300 + k, backward_seed=400 + k,
                              target=torch.full((cam.height, cam.width, 3), 0.3, device="cuda"),
                              g_textures=[torch.zeros_like(t) for t in ds.textures],
                              g_roughness=torch.zeros_like(ds.roughness)))
    return abi, scenes, jobs


def _reset(jobs):
    for j in jobs:
        j.image.zero_()
        for g in j.g_textures:
            g.zero_()
        j.g_roughness.zero_()


def _snapshot(jobs):
    return [(j.image.clone(), [g.clone() for g in j.g_textures], j.g_roughness.clone()) for j in jobs]


def test_noalloc_batch_matches_allocating_batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi, scenes, jobs = _setup()
    opts = abi.pt_batch_opts(4, 4, 4, 128)
    stream = torch.cuda.current_stream().cuda_stream
    _reset(jobs)
    abi.pt_render_batch([j.struct() for j in jobs], opts, stream)
    torch.cuda.synchronize()
    want = _snapshot(jobs)
    for call in range(2):
        _reset(jobs)
        abi.pt_render_batch_noalloc([j.struct() for j in jobs], opts, stream)
        torch.cuda.synchronize()
        for j, (img, gts, gr) in zip(jobs, want):
            assert torch.allclose(j.image, img, rtol=1e-6, atol=0), call
            for g, e in zip(j.g_textures, gts):
                cos = float((g * e).sum() / (g.norm() * e.norm() + 1e-30))
                assert cos > 0.9999, (call, cos)
            assert torch.allclose(j.g_roughness, gr, rtol=1e-3, atol=1e-7), call
        assert float(sum(j.g_roughness.abs().sum() for j in jobs)) > 0


def test_noalloc_rejects_requests_beyond_its_limits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi, scenes, jobs = _setup()
    too_many = [jobs[0].struct()] * 65            # PT_NOALLOC_MAX_JOBS = 64
    with pytest.raises(abi.PtError) as e:
        abi.pt_render_batch_noalloc(too_many, abi.pt_batch_opts(4, 4, 4, 128))
    assert e.value.code == abi.PT_ERR_ARG
    one_px_tiles = abi.pt_batch_opts(1, 4, 4, 128)
    many = [jobs[1].struct()] * 40              # 40 jobs x 64*32 one-pixel tiles = 81,920 > PT_NOALLOC_MAX_ITEMS
    with pytest.raises(abi.PtError) as e:
        abi.pt_render_batch_noalloc(many, one_px_tiles)
    assert e.value.code == abi.PT_ERR_ARG
