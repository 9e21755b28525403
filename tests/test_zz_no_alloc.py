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
        if j.g_env is not None:
            j.g_env.zero_()


def _snapshot(jobs):
    return [(j.image.clone(), [g.clone() for g in j.g_textures], j.g_roughness.clone(),
             None if j.g_env is None else j.g_env.clone()) for j in jobs]


def _cos(g, e):
    return float((g * e).sum() / (g.norm() * e.norm() + 1e-30))


def _check(jobs, want, tag):
    for j, (img, gts, gr, ge) in zip(jobs, want):
        assert torch.allclose(j.image, img, rtol=1e-6, atol=0), tag
        for g, e in zip(j.g_textures, gts):
            assert _cos(g, e) > 0.9999, (tag, _cos(g, e))
        assert torch.allclose(j.g_roughness, gr, rtol=1e-3, atol=1e-7), tag
        if ge is not None:
            assert float(ge.abs().sum()) > 0
            assert _cos(j.g_env, ge) > 0.9999, (tag, _cos(j.g_env, ge))


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
        _check(jobs, want, call)
        assert float(sum(j.g_roughness.abs().sum() for j in jobs)) > 0


def test_noalloc_small_call_after_large_and_env_gradients():
    """A one-job call with a small image after the three-job call must not pick up
    the larger call's job table or work lists left in the shared array; a job
    with environment-map gradients takes the env-gradient kernel variant.  Once
    warmed up, a call leaves the device's free memory unchanged."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import batch
    abi, scenes, jobs = _setup()
    opts = abi.pt_batch_opts(4, 4, 4, 128)
    stream = torch.cuda.current_stream().cuda_stream
    ds = scenes[1]
    small = batch.Job(ds, S.Camera((0.5, 2.0, 6.0), (0.0, 0.4, 0.0), (0.0, 1.0, 0.0), 45.0, 9, 7), 4,
                      seed=77, backward_seed=78, target=torch.full((7, 9, 3), 0.2, device="cuda"),
                      g_textures=[torch.zeros_like(t) for t in ds.textures],
                      g_roughness=torch.zeros_like(ds.roughness),
                      g_env=torch.zeros((ds.scene.env.shape[0], ds.scene.env.shape[1], 4), device="cuda"))
    _reset([small])
    abi.pt_render_batch([small.struct()], opts, stream)
    torch.cuda.synchronize()
    want = _snapshot([small])
    for _ in range(2):                      # large call, then the small one
        abi.pt_render_batch_noalloc([j.struct() for j in jobs], opts, stream)
        _reset([small])
        abi.pt_render_batch_noalloc([small.struct()], opts, stream)
        torch.cuda.synchronize()
        _check([small], want, "small after large")
    free0, _ = torch.cuda.mem_get_info()
    abi.pt_render_batch_noalloc([j.struct() for j in jobs], opts, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_a_capturing_stream():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    abi, scenes, jobs = _setup()
    opts = abi.pt_batch_opts(4, 4, 4, 128)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g, stream=s):
        try:
            abi.pt_render_batch_noalloc([j.struct() for j in jobs], opts, s.cuda_stream)
        except abi.PtError as e:
            codes.append(e.code)
    assert codes == [abi.PT_ERR_STATE]


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
