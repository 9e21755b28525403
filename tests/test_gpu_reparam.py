"""GPU parity of reparameterized PRB (translation gradients, Sec. 4.7) vs the FP64 oracle.

The CUDA kernel computes the gradients in reverse mode (PRB replay, closed-form
warp-field coefficients); the oracle computes the same estimator in forward mode
(chart dual numbers for the warp divergence).  Same seeds, same options, same
auxiliary random numbers.  FP32 against FP64 can flip an auxiliary ray's hit at a
triangle edge, so the comparison is on the accumulated gradient vector.
"""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

from parity import cosine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_01284_gb300 import abi
    abi.load()
    return abi


def _compare(oracle_mod, sc, spp, max_depth, seed, gi, rr_depth=-1, layout=1, **opts):
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    cam = sc.cameras[0]
    ds = DeviceScene(sc, layout=layout)
    st = RenderSettings(width=cam.width, height=cam.height, spp=spp, max_depth=max_depth, rr_depth=rr_depth,
                        seed=seed)
    g = torch.zeros((sc.n_shapes, 3), device="cuda")
    rays = torch.zeros(1, dtype=torch.int64, device="cuda")
    ds.backward_reparam(st, torch.as_tensor(gi[None], dtype=torch.float32, device="cuda"), g, rays=rays, **opts)
    torch.cuda.synchronize()
    assert ds.status() == 0
    r = oracle_mod.render_in(cam, spp, max_depth, seed, rr_depth, True)
    g_ref, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, gi, **opts)
    gg = g.cpu().numpy().astype(np.float64)
    c = cosine(gg.ravel(), g_ref.ravel())
    rel = np.abs(gg - g_ref).max() / np.abs(g_ref).max()
    print(f"{sc.name}: cosine {c:.7f} max rel {rel:.2e} rays {int(rays.item())}\n gpu {gg.ravel()}\n ref {g_ref.ravel()}")
    return gg, g_ref, c, rel, int(rays.item())


def test_reparam_parity_shadow_scene(lib, oracle_mod):
    sc = S.shadow_scene()
    gi = np.random.default_rng(2).random((64, 64, 3)) + 0.5
    gg, g_ref, c, rel, rays = _compare(oracle_mod, sc, 16, 3, 21, gi)
    assert c >= 0.99999
    assert rel < 1e-4  # measured 4e-6
    assert rays > 64 * 64 * 16


@pytest.mark.parametrize("border", [0.0, 4.0])
def test_reparam_parity_camera_rays(lib, oracle_mod, border):
    """Camera-ray warps only (black occluder over a uniform sky) across the right image
    border: the flux through the image-border edges, or (option) the border window."""
    sc = S.occluder_sky(center=(0.5, 0.2), side=0.6)
    gi = np.random.default_rng(3).random((64, 64, 3))
    _, _, c, rel, _ = _compare(oracle_mod, sc, 16, 2, 5, gi, border=border)
    assert c >= 0.99999
    assert rel < 1e-4  # measured 9e-6 with the window


def test_reparam_parity_cornell_multibounce(lib, oracle_mod):
    """Six shapes, indirect bounces, no jackknife and other options: every path vertex warps."""
    sc = S.cornell(width=48, height=48)
    gi = np.random.default_rng(4).random((48, 48, 3))
    _, _, c, rel, _ = _compare(oracle_mod, sc, 4, 4, 9, gi, layout=0, n_aux=8, kappa=2000.0, jackknife=0,
                               power=4.0)
    assert c >= 0.99999
    assert rel < 1e-3  # measured 5e-5
    _, _, c, rel, _ = _compare(oracle_mod, sc, 4, 4, 9, gi, rr_depth=2)
    assert c >= 0.99999
    assert rel < 1e-3


def test_reparam_arguments(lib):
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=16, height=16)
    ds = DeviceScene(sc)
    st = RenderSettings(width=16, height=16, spp=2, max_depth=2, rr_depth=-1, seed=1)
    gi = torch.ones((1, 16, 16, 3), device="cuda")
    g = torch.zeros((3, 3), device="cuda")
    for bad in (dict(n_aux=1), dict(n_aux=33), dict(kappa=0.0), dict(kernel_scale=0.5), dict(eps=0.0),
                dict(miss=-1.0), dict(border=-1.0), dict(jackknife=2), dict(power=-1.0), dict(edge_spp=-1),
                dict(edge_spp=4097)):
        with pytest.raises(lib.PtError):
            ds.backward_reparam(st, gi, g, **bad)
    with pytest.raises(ValueError):
        ds.backward_reparam(st, gi, torch.zeros((2, 3), device="cuda"))
    from dataclasses import replace
    with pytest.raises(lib.PtError):
        ds.backward_reparam(replace(st, block_size=256), gi, g)
    # zero loss gradient: nothing is accumulated
    ds.backward_reparam(st, torch.zeros_like(gi), g)
    torch.cuda.synchronize()
    assert not g.any()


def test_reparam_pixel_edge_term_parity(lib, oracle_mod):
    """The pixel-edge term on its own (gradient with edge paths minus without), in
    translation and vertex mode, on the whole image and on a ragged crop whose border
    edges count for the inside pixel only."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.occluder_sky(center=(0.15, 0.1), side=0.8, width=40, height=40)
    cam = sc.cameras[0]
    osc = oracle_mod.OracleScene(sc)
    ds = DeviceScene(sc)
    for crop in (None, (5, 7, 27, 22)):
        h, w = (40, 40) if crop is None else (crop[3], crop[2])
        gi = np.random.default_rng(11).random((h, w, 3)) - 0.5
        st = RenderSettings(width=40, height=40, spp=4, max_depth=2, rr_depth=-1, seed=31, crop=crop)
        r = oracle_mod.render_in(cam, 4, 2, 31, -1, True, crop=crop)
        gim = torch.as_tensor(gi[None], dtype=torch.float32, device="cuda")
        n_edges = 41 * 40 * 2 if crop is None else 28 * 22 + 23 * 27
        for vertex in (False, True):
            got, ref, n_rays = [], [], []
            for edge_spp in (0, 8):
                gt = torch.zeros((sc.n_shapes, 3), device="cuda")
                gv = torch.zeros((sc.n_tris, 3, 3), device="cuda") if vertex else None
                rays = torch.zeros(1, dtype=torch.int64, device="cuda")
                ds.backward_reparam(st, gim, gt, g_vertices=gv, rays=rays, edge_spp=edge_spp)
                torch.cuda.synchronize()
                assert ds.status() == 0
                got.append((gv if vertex else gt).cpu().numpy().astype(np.float64))
                ref.append(oracle_mod.grad_reparam(osc, r, gi, vertex=vertex, edge_spp=edge_spp)[0])
                n_rays.append(int(rays.item()))
            assert n_rays[1] - n_rays[0] >= n_edges * 8  # at least the camera ray of every edge path
            d, dr = got[1] - got[0], ref[1] - ref[0]
            c = cosine(d.ravel(), dr.ravel())
            rel = np.abs(d - dr).max() / np.abs(dr).max()
            print(f"edge term crop={crop} vertex={vertex}: cosine {c:.7f} max rel {rel:.2e}, "
                  f"{np.abs(dr).max() / np.abs(ref[0]).max():.2f} of the interior terms")
            assert c >= 0.9999 and rel < 1e-3


def test_reparam_fullsize_crop_parity(lib, oracle_mod):
    """The bench's launch: 196,608-triangle sphere scene (33 shapes), 1024x1024, 16 spp,
    depth 8, roulette from 3, wide BVH, whole-image launch.  dLoss/dI is non-zero on two
    16x16 crops only, so the oracle's crops and the GPU's full image differentiate the
    same sum."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.spheres()
    ds = DeviceScene(sc, layout=lib.PT_BVH_WIDE)
    st = RenderSettings(width=1024, height=1024, spp=16, max_depth=8, rr_depth=3, seed=12)
    crops = [(400, 540, 16, 16), (600, 600, 16, 16)]
    rng = np.random.default_rng(8)
    gi = np.zeros((1024, 1024, 3), np.float32)
    osc = oracle_mod.OracleScene(sc)
    g_ref = np.zeros((sc.n_shapes, 3))
    for (x0, y0, w, h) in crops:
        g = rng.random((h, w, 3)).astype(np.float32)
        gi[y0:y0 + h, x0:x0 + w] = g
        r = oracle_mod.render_in(sc.cameras[0], 16, 8, 12, 3, True, crop=(x0, y0, w, h))
        g_ref += oracle_mod.grad_reparam(osc, r, g)[0]
    gt = torch.zeros((sc.n_shapes, 3), device="cuda")
    ds.backward_reparam(st, torch.as_tensor(gi[None], device="cuda"), gt)
    torch.cuda.synchronize()
    assert ds.status() == 0
    gg = gt.cpu().numpy().astype(np.float64)
    c = cosine(gg.ravel(), g_ref.ravel())
    rel = np.abs(gg - g_ref).max() / np.abs(g_ref).max()
    print(f"full-size reparam: cosine {c:.7f} max rel {rel:.2e}")
    assert c >= 0.9999
    assert rel < 1e-2


def test_reparam_recovers_occluder_position(lib):
    """Gradient descent on the occluder's translation through the autograd wrapper:
    the shadow of a target render pulls it back (a non-reparameterized derivative
    would be zero here)."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings, render_translated
    sc = S.shadow_scene(width=48, height=48)
    truth = np.zeros((3, 3))
    truth[2] = (0.15, 0.0, -0.08)
    st_t = RenderSettings(width=48, height=48, spp=256, max_depth=2, rr_depth=-1, seed=99)
    target = DeviceScene(sc.translated(truth)).forward(st_t)
    t = torch.zeros((3, 3), device="cuda", requires_grad=True)
    opt = torch.optim.Adam([t], lr=0.01)
    mask = torch.zeros((3, 3), device="cuda")
    mask[2] = 1.0
    for k in range(80):
        st = RenderSettings(width=48, height=48, spp=16, max_depth=2, rr_depth=-1, seed=1000 + k,
                            backward_seed=5000 + k)
        opt.zero_grad()
        img = render_translated(sc, st, t)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        t.grad *= mask
        opt.step()
    err = (t.detach().cpu().numpy() - truth)[2]
    print("recovered", t.detach().cpu().numpy()[2], "truth", truth[2], "loss", loss.item())
    assert np.abs(err[[0, 2]]).max() < 0.03   # started 0.15 / 0.08 away
    assert abs(err[1]) < 0.05


def test_reparam_two_cameras_crop_and_lanes(lib, oracle_mod):
    """Two cameras in one call, a ragged crop and every lane split: the gradient of the
    call is the sum of the oracle's per-camera crops."""
    from dataclasses import replace
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=40, height=30)
    cam2 = S.Camera((1.2, 1.4, 1.0), (-0.4, 0.0, 0.0), (0.0, 1.0, 0.0), 50.0, 40, 30)
    ds = DeviceScene(sc, layout=0)
    crop = (5, 3, 29, 21)
    gi = np.random.default_rng(7).random((2, 21, 29, 3)).astype(np.float32)
    osc = oracle_mod.OracleScene(sc)
    g_ref = np.zeros((3, 3))
    for ci, cam in enumerate((sc.cameras[0], cam2)):
        r = oracle_mod.render_in(cam, 6, 3, 13, 2, True, cam_index=ci, crop=crop)
        g_ref += oracle_mod.grad_reparam(osc, r, gi[ci])[0]
    base = RenderSettings(width=40, height=30, spp=6, max_depth=3, rr_depth=2, seed=13, crop=crop)
    for lanes in (1, 2, 4, 8):
        g = torch.zeros((3, 3), device="cuda")
        ds.backward_reparam(replace(base, lanes_per_pixel=lanes), torch.as_tensor(gi, device="cuda"), g,
                            cams=[sc.cameras[0], cam2])
        torch.cuda.synchronize()
        gg = g.cpu().numpy().astype(np.float64)
        rel = np.abs(gg - g_ref).max() / np.abs(g_ref).max()
        print("lanes", lanes, "max rel", rel)
        assert rel < 1e-3


def _compare_vertices(oracle_mod, sc, spp, max_depth, seed, gi, rr_depth=-1, layout=1, **opts):
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    cam = sc.cameras[0]
    ds = DeviceScene(sc, layout=layout)
    st = RenderSettings(width=cam.width, height=cam.height, spp=spp, max_depth=max_depth, rr_depth=rr_depth,
                        seed=seed)
    gv = torch.zeros((sc.n_tris, 3, 3), device="cuda")
    gt = torch.zeros((sc.n_shapes, 3), device="cuda")
    gim = torch.as_tensor(gi[None], dtype=torch.float32, device="cuda")
    ds.backward_reparam(st, gim, gt, g_vertices=gv, **opts)
    torch.cuda.synchronize()
    assert ds.status() == 0
    r = oracle_mod.render_in(cam, spp, max_depth, seed, rr_depth, True)
    ref, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, gi, vertex=True, **opts)
    g = gv.cpu().numpy().astype(np.float64)
    c = cosine(g.ravel(), ref.ravel())
    rel = np.abs(g - ref).max() / np.abs(ref).max()
    sums = np.zeros((sc.n_shapes, 3))
    for t in range(sc.n_tris):
        sums[sc.tri_shape[t]] += g[t].sum(axis=0)
    gtn = gt.cpu().numpy().astype(np.float64)
    srel = np.abs(sums - gtn).max() / np.abs(gtn).max()
    print(f"{sc.name} vertices: cosine {c:.7f} max rel {rel:.2e}; corner sums vs translation {srel:.2e}")
    return c, rel, srel


def test_reparam_vertex_parity(lib, oracle_mod):
    gi = np.random.default_rng(2).random((48, 48, 3)) + 0.5
    c, rel, srel = _compare_vertices(oracle_mod, S.shadow_scene(width=48, height=48), 8, 3, 21, gi)
    assert c >= 0.99999 and rel < 1e-3 and srel < 1e-4
    gi = np.random.default_rng(3).random((48, 48, 3))
    c, rel, srel = _compare_vertices(oracle_mod, S.occluder_sky(center=(0.5, 0.2), side=0.6, width=48, height=48),
                                     8, 2, 5, gi)
    assert c >= 0.99999 and rel < 1e-3 and srel < 1e-4
    gi = np.random.default_rng(4).random((24, 24, 3))
    c, rel, srel = _compare_vertices(oracle_mod, S.cornell(width=24, height=24), 2, 4, 9, gi, layout=0,
                                     jackknife=0, n_aux=8)
    assert c >= 0.9999 and rel < 1e-2 and srel < 1e-3


@pytest.mark.parametrize("bsdf", [S.BSDF_CONDUCTOR, S.BSDF_BLEND])
def test_reparam_glossy_parity(lib, oracle_mod, bsdf):
    """Glossy floor (GGX conductor, blend): the rays leaving it add the BSDF's
    directional terms, and the arriving ray's warp takes the floor's incident-direction
    terms (posted one vertex later); in vertex mode the BSDF value also follows the
    floor triangles' turning normals (closed form on the GPU, dual-number frame in the
    oracle)."""
    gi = np.random.default_rng(5).random((48, 48, 3)) + 0.2
    sc = S.shadow_scene(width=48, height=48, floor_bsdf=bsdf, floor_alpha=0.3)
    _, _, c, rel, _ = _compare(oracle_mod, sc, 16, 3, 31, gi)
    assert c >= 0.99999 and rel < 1e-3
    c, rel, srel = _compare_vertices(oracle_mod, sc, 8, 3, 31, gi)
    assert c >= 0.9999 and rel < 5e-3 and srel < 1e-4


def test_reparam_textured_blend_scene(lib, oracle_mod):
    """96-shape Cornell room (textured blend BSDFs with per-shape roughness), roulette."""
    sc = S.cornell96(width=32, height=32, tex_res=256)
    gi = np.random.default_rng(6).random((32, 32, 3))
    _, _, c, rel, _ = _compare(oracle_mod, sc, 2, 4, 17, gi, rr_depth=2, layout=0, n_aux=8)
    assert c >= 0.9999 and rel < 1e-2
    c, rel, srel = _compare_vertices(oracle_mod, sc, 2, 4, 17, gi, rr_depth=2, layout=0, n_aux=8)
    assert c >= 0.999 and srel < 1e-3


def test_reparam_without_light_sampling_and_depth_one(lib, oracle_mod):
    """BSDF sampling only (no light-sample rays) on the blend floor, and depth 1 (the
    directly visible sky: camera warps only)."""
    gi = np.random.default_rng(9).random((32, 32, 3))
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    for sc, nee, depth in ((S.shadow_scene(width=32, height=32, floor_bsdf=S.BSDF_BLEND), False, 3),
                           (S.occluder_sky(width=32, height=32), True, 1)):
        ds = DeviceScene(sc, layout=1)
        n = sc.n_shapes
        st = RenderSettings(width=32, height=32, spp=16, max_depth=depth, rr_depth=-1, seed=4, nee=nee)
        g = torch.zeros((n, 3), device="cuda")
        ds.backward_reparam(st, torch.as_tensor(gi[None], dtype=torch.float32, device="cuda"), g)
        torch.cuda.synchronize()
        r = oracle_mod.render_in(sc.cameras[0], 16, depth, 4, -1, nee)
        ref, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, gi)
        gg = g.cpu().numpy().astype(np.float64)
        scale = max(np.abs(ref).max(), 1e-6)
        rel = np.abs(gg - ref).max() / scale
        print(f"nee={nee} depth={depth}: max rel {rel:.2e}, |g| {np.abs(ref).max():.3g}")
        assert np.abs(ref).max() > 1.0 and rel < 1e-3


def _blur(img, sigma=1.5):
    """Gaussian blur of [1, H, W, 3] images (separable, zero padding)."""
    r = int(3 * sigma)
    x = torch.arange(-r, r + 1, device=img.device, dtype=torch.float32)
    k = torch.exp(-0.5 * (x / sigma) ** 2)
    k = k / k.sum()
    t = img.permute(0, 3, 1, 2).reshape(-1, 1, img.shape[1], img.shape[2])
    t = torch.nn.functional.conv2d(t, k.view(1, 1, 1, -1), padding=(0, r))
    t = torch.nn.functional.conv2d(t, k.view(1, 1, -1, 1), padding=(r, 0))
    return t.reshape(img.shape[0], 3, img.shape[1], img.shape[2]).permute(0, 2, 3, 1)


def test_reparam_recovers_square_scale_through_vertices(lib):
    """Vertex positions as a torch expression of one scale parameter: the square's
    corners are c + s (p - c); 60 Adam steps on s through render_vertices recover a
    1.25x larger square from its target image (the derivative flows through every
    corner's gradient).  The loss compares Gaussian-blurred images: with the box
    pixel filter, a warp moves samples across pixel edges without moving their
    pixel, and a loss gradient that changes sign from one pixel to the next (the
    plain L2 loss on a one-pixel-wide ring) can turn those edge terms into the
    dominant ones; a blur of 1.5 pixels makes dLoss/dI smooth."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings, render_vertices
    sc = S.occluder_sky(width=48, height=48)
    base = torch.as_tensor(sc.vertices, dtype=torch.float32, device="cuda")
    c = torch.tensor([0.15, 0.1, -3.0], device="cuda")
    true_s = 1.25
    target_sc = S.occluder_sky(width=48, height=48, side=0.4 * true_s)
    target = DeviceScene(target_sc).forward(RenderSettings(width=48, height=48, spp=256, max_depth=2, seed=99))
    s = torch.ones(1, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([s], lr=0.02)
    for k in range(60):
        st = RenderSettings(width=48, height=48, spp=16, max_depth=2, seed=100 + k, backward_seed=500 + k)
        opt.zero_grad()
        img = render_vertices(sc, st, c + s * (base - c))
        loss = ((_blur(img) - _blur(target)) ** 2).mean()
        loss.backward()
        opt.step()
    print("recovered scale", s.item(), "truth", true_s)
    assert abs(s.item() - true_s) < 0.03


def test_reparam_recovers_square_scale_with_a_sharp_loss(lib):
    """The same scale recovery with the plain per-pixel L2 loss, no blur: the
    pixel-edge term gives the derivative of the box-filtered pixels themselves, so
    the loss on a one-pixel-wide ring of disagreement pulls the right way."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings, render_vertices
    sc = S.occluder_sky(width=48, height=48)
    base = torch.as_tensor(sc.vertices, dtype=torch.float32, device="cuda")
    c = torch.tensor([0.15, 0.1, -3.0], device="cuda")
    true_s = 1.25
    target_sc = S.occluder_sky(width=48, height=48, side=0.4 * true_s)
    target = DeviceScene(target_sc).forward(RenderSettings(width=48, height=48, spp=256, max_depth=2, seed=99))
    s = torch.ones(1, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([s], lr=0.02)
    for k in range(60):
        st = RenderSettings(width=48, height=48, spp=16, max_depth=2, seed=100 + k, backward_seed=500 + k)
        opt.zero_grad()
        img = render_vertices(sc, st, c + s * (base - c), edge_spp=4)
        loss = ((img - target) ** 2).mean()
        loss.backward()
        opt.step()
    print("recovered scale (sharp loss)", s.item(), "truth", true_s)
    assert abs(s.item() - true_s) < 0.03


def test_reparam_camera_translation(lib, oracle_mod):
    """render_translated with a camera offset: its gradient is minus the sum of all
    shapes' translation gradients (parity with the oracle's), and gradient descent on
    the offset recovers a moved camera from its image alone.  Everything in view
    slides when the camera moves, so this leans on the flux through the image-border
    edges of the pixel-edge term."""
    from paper_2202_01284_gb300.render import RenderSettings, render_translated
    sc = S.shadow_scene(width=48, height=48)
    st = RenderSettings(width=48, height=48, spp=8, max_depth=3, rr_depth=-1, seed=21)
    gi = np.random.default_rng(9).random((48, 48, 3))
    off = torch.zeros(3, device="cuda", requires_grad=True)
    img = render_translated(sc, st, camera_offset=off)
    (img * torch.as_tensor(gi[None], dtype=torch.float32, device="cuda")).sum().backward()
    r = oracle_mod.render_in(sc.cameras[0], 8, 3, 21, -1, True)
    g_ref = -oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, gi)[0].sum(axis=0)
    got = off.grad.cpu().numpy().astype(np.float64)
    rel = np.abs(got - g_ref).max() / np.abs(g_ref).max()
    print("camera offset gradient", got, "oracle", g_ref, "max rel", rel)
    assert rel < 1e-3

    truth = np.array([-0.08, 0.06, 0.1])
    tsc = sc.camera_moved(truth)
    from paper_2202_01284_gb300.render import DeviceScene
    target = DeviceScene(tsc).forward(RenderSettings(width=48, height=48, spp=256, max_depth=2, seed=99))
    off = torch.zeros(3, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([off], lr=0.01)
    for k in range(60):
        if k == 40:
            for grp in opt.param_groups:
                grp["lr"] = 0.003
        st = RenderSettings(width=48, height=48, spp=16, max_depth=2, seed=1000 + k, backward_seed=5000 + k)
        opt.zero_grad()
        loss = ((render_translated(sc, st, camera_offset=off, edge_spp=4) - target) ** 2).mean()
        loss.backward()
        opt.step()
    err = off.detach().cpu().numpy() - truth
    print("recovered camera offset", off.detach().cpu().numpy(), "truth", truth, "loss", loss.item())
    assert np.abs(err).max() < 0.03   # started 0.1 away; measured 0.015


@pytest.mark.parametrize("n_aux", [2, 5, 32])
def test_reparam_auxiliary_group_sizes(lib, oracle_mod, n_aux):
    """Lobes of 2, 5 (groups of 8 lanes with 3 idle) and 32 auxiliary rays (one
    lobe per warp round), jackknife on, vertex mode too."""
    sc = S.shadow_scene(width=32, height=32)
    gi = np.random.default_rng(12).random((32, 32, 3)) + 0.1
    _, _, c, rel, _ = _compare(oracle_mod, sc, 4, 3, 41, gi, n_aux=n_aux)
    assert c >= 0.99999 and rel < 1e-3
    c, rel, srel = _compare_vertices(oracle_mod, sc, 4, 3, 41, gi, n_aux=n_aux)
    assert c >= 0.9999 and rel < 5e-3 and srel < 1e-4


def test_reparam_crops_on_the_image_border(lib, oracle_mod):
    """Ragged crops that touch the image's corners: their outer edges lie on the image
    border (flux through it), their inner edges count for the inside pixel only; the
    four crops' gradients sum to the whole image's."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=40, height=30)
    ds = DeviceScene(sc, layout=0)
    osc = oracle_mod.OracleScene(sc)
    gi_full = np.random.default_rng(13).random((30, 40, 3)) - 0.3
    crops = [(0, 0, 17, 13), (17, 0, 23, 13), (0, 13, 17, 17), (17, 13, 23, 17)]
    g_sum = np.zeros((3, 3))
    for crop in crops:
        x0, y0, w, h = crop
        gi = np.ascontiguousarray(gi_full[y0:y0 + h, x0:x0 + w])
        st = RenderSettings(width=40, height=30, spp=4, max_depth=3, rr_depth=-1, seed=23, crop=crop)
        g = torch.zeros((3, 3), device="cuda")
        ds.backward_reparam(st, torch.as_tensor(gi[None], dtype=torch.float32, device="cuda"), g, edge_spp=2)
        torch.cuda.synchronize()
        assert ds.status() == 0
        r = oracle_mod.render_in(sc.cameras[0], 4, 3, 23, -1, True, crop=crop)
        ref = oracle_mod.grad_reparam(osc, r, gi, edge_spp=2)[0]
        gg = g.cpu().numpy().astype(np.float64)
        rel = np.abs(gg - ref).max() / np.abs(ref).max()
        print("crop", crop, "max rel", rel)
        assert rel < 1e-3
        g_sum += gg
    st = RenderSettings(width=40, height=30, spp=4, max_depth=3, rr_depth=-1, seed=23)
    g = torch.zeros((3, 3), device="cuda")
    ds.backward_reparam(st, torch.as_tensor(gi_full[None], dtype=torch.float32, device="cuda"), g, edge_spp=2)
    torch.cuda.synchronize()
    whole = g.cpu().numpy().astype(np.float64)
    print("sum of the crops", g_sum.ravel(), "whole image", whole.ravel())
    assert np.abs(g_sum - whole).max() < 1e-4 * np.abs(whole).max()
