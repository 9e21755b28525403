"""The batched persistent launch at its full workload against the FP64 oracle.

64 cameras of uneven size (128..1024 per side, 4..64 spp) over the three procedural
scenes of about 10k, 200k and 2M triangles, forward + PRB adjoint in one persistent
launch: once replayed from a captured CUDA graph (Batch), once through
pt_render_batch.  For one job of each scene the oracle renders a 16x16 crop with the
job's seed (image parity, path-divergence outliers counted through the GPU's
decision fingerprints of the same crop) and differentiates it with the job's
backward seed.  For the gradients the target of those three jobs equals the batch's
own image outside the crop (the batch kernel is deterministic, so dLoss/dI is
exactly zero there) and differs inside it: the batch's texture and roughness
gradients then differentiate the same function as the oracle's tape on the crop.
"""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import GRAD_COSINE, PIXEL_FRACTION, cosine, rel_ok

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def c4():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi, batch, render
    abi.load()
    scenes = S.batch_scenes()
    dss = [render.DeviceScene(sc, layout=abi.PT_BVH_WIDE) for sc in scenes]
    cams = S.batch_cameras(64, 3)
    jobs = []
    for k, bc in enumerate(cams):
        ds = dss[bc.scene]
        jobs.append(batch.Job(ds, bc.camera, bc.spp, seed=1000 + k, backward_seed=2000 + k,
                              target=torch.full((bc.camera.height, bc.camera.width, 3), 0.3, device="cuda"),
                              g_textures=[torch.zeros_like(t) for t in ds.textures],
                              g_roughness=torch.zeros_like(ds.roughness)))
    picks = [next(k for k, bc in enumerate(cams) if bc.scene == s) for s in range(3)]
    return abi, batch, render, scenes, dss, cams, jobs, picks


def _crop_of(cam):
    # the image centre looks at the spheres (every camera aims at their middle)
    return (cam.width // 2 - 8, cam.height // 2 - 8, 16, 16)


def _zero(jobs):
    for j in jobs:
        for g in j.g_textures:
            g.zero_()
        j.g_roughness.zero_()


def test_c4_graph_batch_forward_matches_oracle(c4, oracle_mod):
    from dataclasses import replace
    abi, batch, render, scenes, dss, cams, jobs, picks = c4
    b = batch.Batch(jobs, tile=8, lanes_per_pixel=8, ctas_per_sm=4)
    b.capture()
    _zero(jobs)
    b.replay()
    torch.cuda.synchronize()
    assert all(ds.status() == 0 for ds in dss)
    all_ok, all_n, divergent = 0, 0, 0
    for k in picks:
        bc, j = cams[k], jobs[k]
        crop = _crop_of(bc.camera)
        x0, y0, w, h = crop
        sc = scenes[bc.scene]
        r = oracle_mod.render_in(bc.camera, bc.spp, 8, 1000 + k, 3, True, crop=crop)
        ref, _, refh = oracle_mod.render(oracle_mod.OracleScene(sc), r, per_sample=True)
        st = render.RenderSettings(width=bc.camera.width, height=bc.camera.height, spp=bc.spp, max_depth=8,
                                   rr_depth=3, seed=1000 + k, crop=crop)
        _, _, gh = dss[bc.scene].forward(st, cams=[bc.camera], per_sample=True)
        clean = (gh[0].cpu().numpy().view(np.uint32) == refh.astype(np.uint32)).all(axis=-1)
        img = j.image[y0:y0 + h, x0:x0 + w].cpu().numpy()
        ok = rel_ok(img, ref).all(axis=-1)
        print(f"job {k} scene {sc.n_tris} tris {bc.camera.width}x{bc.camera.height} {bc.spp} spp: "
              f"clean {clean.mean():.4f} ok on clean {ok[clean].mean():.4f} ok all {ok.mean():.4f}")
        assert ok[clean].mean() >= PIXEL_FRACTION
        all_ok += int(ok.sum())
        all_n += ok.size
        divergent += int((~clean).sum())
    print(f"C4 forward: all pixels {all_ok / all_n:.5f}, divergent {divergent} of {all_n}")
    assert all_ok / all_n >= 0.99
    b.close()


def test_c4_batch_gradients_match_oracle(c4, oracle_mod):
    abi, batch, render, scenes, dss, cams, jobs, picks = c4
    opts = abi.pt_batch_opts(8, 8, 4, 128)
    stream = torch.cuda.current_stream().cuda_stream
    # first launch: the images; then targets equal to them outside the crops
    abi.pt_render_batch([j.struct() for j in jobs], opts, stream)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    n_div = 0
    for k in picks:
        bc, j = cams[k], jobs[k]
        crop = _crop_of(bc.camera)
        x0, y0, w, h = crop
        # pixels whose samples all take the oracle's decisions with the backward seed
        # (the adjoint replays those paths); the others get target = image, i.e. no
        # gradient on either side (a flipped texel or triangle choice between FP32 and
        # FP64 moves whole gradient terms)
        r = oracle_mod.render_in(bc.camera, bc.spp, 8, 2000 + k, 3, True, crop=crop)
        _, _, refh = oracle_mod.render(oracle_mod.OracleScene(scenes[bc.scene]), r, per_sample=True)
        st = render.RenderSettings(width=bc.camera.width, height=bc.camera.height, spp=bc.spp, max_depth=8,
                                   rr_depth=3, seed=2000 + k, crop=crop)
        _, _, gh = dss[bc.scene].forward(st, cams=[bc.camera], per_sample=True)
        clean = (gh[0].cpu().numpy().view(np.uint32) == refh.astype(np.uint32)).all(axis=-1)
        n_div += int((~clean).sum())
        noise = rng.uniform(-0.2, 0.2, (h, w, 3)).astype(np.float32) * clean[..., None]
        t = j.image.clone()
        t[y0:y0 + h, x0:x0 + w] += torch.as_tensor(noise, device="cuda")
        j.target.copy_(t)
    print(f"divergent pixels excluded from the gradient comparison: {n_div} of {16 * 16 * len(picks)}")
    assert n_div <= 0.05 * 16 * 16 * len(picks)
    before = [j.image.clone() for j in jobs]
    _zero(jobs)
    abi.pt_render_batch([j.struct() for j in jobs], opts, stream)
    torch.cuda.synchronize()
    assert all(torch.equal(j.image, b) for j, b in zip(jobs, before))   # deterministic batch kernel
    for k in picks:
        bc, j = cams[k], jobs[k]
        sc = scenes[bc.scene]
        crop = _crop_of(bc.camera)
        x0, y0, w, h = crop
        W, H = bc.camera.width, bc.camera.height
        gi = (2.0 * (j.image - j.target) / (3.0 * W * H))[y0:y0 + h, x0:x0 + w].cpu().numpy().astype(np.float64)
        r = oracle_mod.render_in(bc.camera, bc.spp, 8, 2000 + k, 3, True, crop=crop)
        _, gt_ref, gr_ref = oracle_mod.grad_tape(oracle_mod.OracleScene(sc), r, gi)
        c_t = cosine(j.g_textures[0].cpu().numpy()[..., :3], gt_ref[0][..., :3])
        c_r = cosine(j.g_roughness.cpu().numpy(), gr_ref)
        print(f"job {k} ({sc.n_tris} tris): texture cosine {c_t:.7f}, roughness cosine {c_r:.7f}")
        assert np.abs(gr_ref).sum() + np.abs(gt_ref[0]).sum() > 0
        assert c_t >= GRAD_COSINE and c_r >= GRAD_COSINE
