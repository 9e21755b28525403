"""GPU parity of the forward-mode reparameterized derivative (pt_render_jvp_reparam).

The kernel computes d image / d eps along a direction of shape translations in one
forward pass; the FP64 oracle computes the same per-pixel derivative in forward
mode (one parameter at a time), with the same seeds and auxiliary random numbers.
The forward and reverse modes are the same estimator, so <grad_image, image_dot>
must equal <direction, reverse-mode gradient> for the same seed.
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


def _jvp(sc, st, direction, layout=1, **opts):
    from paper_2202_01284_gb300.render import DeviceScene
    ds = DeviceScene(sc, layout=layout)
    rays = torch.zeros(1, dtype=torch.int64, device="cuda")
    img, dot = ds.jvp_reparam(st, direction, rays=rays, **opts)
    torch.cuda.synchronize()
    assert ds.status() == 0
    return img[0].cpu().numpy().astype(np.float64), dot[0].cpu().numpy().astype(np.float64), int(rays.item())


@pytest.mark.parametrize("name,shape,axis", [("shadow", 2, 0), ("shadow", 1, 1), ("shadow_conductor", 2, 2),
                                             ("occluder_sky_border", 0, 0), ("cornell", 3, 1)])
def test_jvp_reparam_parity_per_pixel(lib, oracle_mod, name, shape, axis):
    """Per-pixel derivative along one shape's translation axis against the oracle's."""
    from paper_2202_01284_gb300.render import RenderSettings
    sc = {"shadow": lambda: S.shadow_scene(width=32, height=32),
          "shadow_conductor": lambda: S.shadow_scene(width=32, height=32, floor_bsdf=S.BSDF_CONDUCTOR),
          "occluder_sky_border": lambda: S.occluder_sky(center=(0.5, 0.2), side=0.6, width=32, height=32),
          "cornell": lambda: S.cornell(width=24, height=24)}[name]()
    cam = sc.cameras[0]
    spp, depth = 8, 3
    d = np.zeros((sc.n_shapes, 3))
    d[shape, axis] = 1.0
    st = RenderSettings(width=cam.width, height=cam.height, spp=spp, max_depth=depth, rr_depth=-1, seed=17)
    img, dot, rays = _jvp(sc, st, d, edge_spp=2)
    r = oracle_mod.render_in(cam, spp, depth, 17, -1, True)
    _, img_ref, dot_ref = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, dot_param=3 * shape + axis, edge_spp=2)
    c = cosine(dot.ravel(), dot_ref.ravel())
    rel = np.abs(dot - dot_ref).max() / np.abs(dot_ref).max()
    print(f"{name} shape {shape} axis {axis}: image max err {np.abs(img - img_ref).max():.2e}, "
          f"image_dot cosine {c:.7f} max rel {rel:.2e}, rays {rays}")
    assert np.abs(img - img_ref).max() < 1e-3 * max(1.0, np.abs(img_ref).max())
    assert c >= 0.9999 and rel < 5e-3


def test_jvp_reparam_matches_reverse_mode(lib):
    """<grad_image, image_dot(direction)> = <direction, reverse gradient(grad_image)>,
    same seed, a direction over all shapes, on a ragged crop with two cameras."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=40, height=30, floor_bsdf=S.BSDF_BLEND)
    cam2 = S.Camera((1.2, 1.4, 1.0), (-0.4, 0.0, 0.0), (0.0, 1.0, 0.0), 50.0, 40, 30)
    ds = DeviceScene(sc)
    crop = (3, 2, 33, 25)
    st = RenderSettings(width=40, height=30, spp=6, max_depth=4, rr_depth=2, seed=29, crop=crop)
    rng = np.random.default_rng(31)
    direction = rng.normal(size=(3, 3))
    gi = rng.random((2, 25, 33, 3)).astype(np.float32) - 0.4
    cams = [sc.cameras[0], cam2]
    _, dot = ds.jvp_reparam(st, direction, cams=cams, edge_spp=3)
    g = torch.zeros((3, 3), device="cuda")
    ds.backward_reparam(st, torch.as_tensor(gi, device="cuda"), g, cams=cams, edge_spp=3)
    torch.cuda.synchronize()
    lhs = float((dot.cpu().numpy().astype(np.float64) * gi).sum())
    rhs = float((g.cpu().numpy().astype(np.float64) * direction).sum())
    print("forward", lhs, "reverse", rhs)
    assert abs(lhs - rhs) < 1e-4 * max(abs(lhs), abs(rhs))


def test_jvp_reparam_arguments(lib):
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=16, height=16)
    ds = DeviceScene(sc)
    st = RenderSettings(width=16, height=16, spp=2, max_depth=2, rr_depth=-1, seed=1)
    with pytest.raises(ValueError):
        ds.jvp_reparam(st, np.zeros((2, 3)))
    with pytest.raises(lib.PtError):
        ds.jvp_reparam(st, np.zeros((3, 3)), n_aux=1)
    _, dot = ds.jvp_reparam(st, np.zeros((3, 3)))
    torch.cuda.synchronize()
    assert not dot.any()


def test_jvp_reparam_translated_occluder_over_a_metallic_floor(lib):
    """The paper's forward-derivative figure in kind: an occluder (out of the
    camera's view) translated over a GGX-conductor floor, whose shadow and
    reflection move.  The reparameterized derivative image against central finite
    differences of renders (8 x 4096 samples per pixel, both blurred by one pixel):
    measured 0.27 relative L2, the same with 32 auxiliary rays (the estimator's
    bias on this receiver, not noise); a derivative that ignores visibility is 0
    here, i.e. 1.0."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=48, height=48, floor_bsdf=S.BSDF_CONDUCTOR, floor_alpha=0.2)
    d = np.zeros((3, 3))
    d[2, 0] = 1.0
    st = RenderSettings(width=48, height=48, spp=4096, max_depth=3, rr_depth=-1, seed=3)
    _, dot = DeviceScene(sc).jvp_reparam(st, d, edge_spp=16)
    h = 0.01
    off = np.zeros((3, 3))
    off[2, 0] = h
    plus, minus = DeviceScene(sc.translated(off)), DeviceScene(sc.translated(-off))
    fd = torch.zeros_like(dot)
    for k in range(8):  # 8 x 4096 samples per pixel, the same random numbers on both sides
        stf = RenderSettings(width=48, height=48, spp=4096, max_depth=3, rr_depth=-1, seed=5 + k)
        fd += (plus.forward(stf) - minus.forward(stf)) / (2 * h * 8)
    torch.cuda.synchronize()

    def blur(x):
        k = torch.tensor([0.0545, 0.2442, 0.4026, 0.2442, 0.0545], device="cuda")
        t = x.permute(0, 3, 1, 2).reshape(-1, 1, x.shape[1], x.shape[2])
        t = torch.nn.functional.conv2d(t, k.view(1, 1, 1, -1), padding=(0, 2))
        t = torch.nn.functional.conv2d(t, k.view(1, 1, -1, 1), padding=(2, 0))
        return t
    err = float((blur(dot) - blur(fd)).norm() / blur(fd).norm())
    print("forward derivative vs finite differences, relative L2 (1-pixel blur):", err)
    assert err < 0.35


@pytest.mark.parametrize("name,tri,corner,axis", [("shadow", 4, 1, 0), ("shadow_conductor", 0, 2, 1),
                                                  ("shadow_conductor", 1, 0, 0), ("occluder_sky_border", 1, 2, 0)])
def test_jvp_reparam_vertices_parity_per_pixel(lib, oracle_mod, name, tri, corner, axis):
    """Vertex mode: the per-pixel derivative along one corner coordinate (a
    non-rigid motion: the triangle's normal turns, which the cosine and a glossy
    floor's BSDF value follow) against the oracle's."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = {"shadow": lambda: S.shadow_scene(width=32, height=32),
          "shadow_conductor": lambda: S.shadow_scene(width=32, height=32, floor_bsdf=S.BSDF_CONDUCTOR),
          "occluder_sky_border": lambda: S.occluder_sky(center=(0.5, 0.2), side=0.6, width=32, height=32)}[name]()
    cam = sc.cameras[0]
    d = np.zeros((sc.n_tris, 3, 3))
    d[tri, corner, axis] = 1.0
    st = RenderSettings(width=cam.width, height=cam.height, spp=8, max_depth=3, rr_depth=-1, seed=19)
    ds = DeviceScene(sc)
    _, dot = ds.jvp_reparam(st, dir_vertices=d, edge_spp=2)
    torch.cuda.synchronize()
    assert ds.status() == 0
    dot = dot[0].cpu().numpy().astype(np.float64)
    r = oracle_mod.render_in(cam, 8, 3, 19, -1, True)
    _, _, ref = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, dot_param=9 * tri + 3 * corner + axis,
                                        vertex=True, edge_spp=2)
    c = cosine(dot.ravel(), ref.ravel())
    rel = np.abs(dot - ref).max() / np.abs(ref).max()
    print(f"{name} triangle {tri} corner {corner} axis {axis}: cosine {c:.7f} max rel {rel:.2e}")
    assert c >= 0.9999 and rel < 5e-3


def test_jvp_reparam_vertices_matches_reverse_mode_and_translations(lib):
    """<grad_image, image_dot(direction)> against the reverse mode's <direction,
    corner gradient> (same seed, glossy blend floor); and moving every corner of
    each shape by that shape's vector gives the translation form's image."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=40, height=30, floor_bsdf=S.BSDF_BLEND)
    ds = DeviceScene(sc)
    st = RenderSettings(width=40, height=30, spp=6, max_depth=4, rr_depth=2, seed=37)
    rng = np.random.default_rng(41)
    dv = rng.normal(size=(sc.n_tris, 3, 3))
    gi = rng.random((1, 30, 40, 3)).astype(np.float32) - 0.4
    _, dot = ds.jvp_reparam(st, dir_vertices=dv, edge_spp=3)
    g = torch.zeros((sc.n_tris, 3, 3), device="cuda")
    gt = torch.zeros((3, 3), device="cuda")
    ds.backward_reparam(st, torch.as_tensor(gi, device="cuda"), gt, g_vertices=g, edge_spp=3)
    torch.cuda.synchronize()
    lhs = float((dot.cpu().numpy().astype(np.float64) * gi).sum())
    rhs = float((g.cpu().numpy().astype(np.float64) * dv).sum())
    print("vertex mode: forward", lhs, "reverse", rhs)
    assert abs(lhs - rhs) < 1e-4 * max(abs(lhs), abs(rhs))
    dt = rng.normal(size=(3, 3))
    _, dot_t = ds.jvp_reparam(st, dt, edge_spp=3)
    _, dot_v = ds.jvp_reparam(st, dir_vertices=np.repeat(dt[sc.tri_shape][:, None, :], 3, axis=1), edge_spp=3)
    torch.cuda.synchronize()
    a, b = dot_t.cpu().numpy(), dot_v.cpu().numpy()
    print("translations as corner motions: max diff", np.abs(a - b).max(), "scale", np.abs(a).max())
    assert np.abs(a - b).max() < 1e-4 * np.abs(a).max()


@pytest.mark.parametrize("vertex", [False, True])
def test_jvp_reparam_random_direction_parity(lib, oracle_mod, vertex):
    """A random direction over every parameter (all shapes, or all corner coordinates:
    the origins of vertex rays move too) against the oracle's derivative along the
    same direction, per pixel."""
    from paper_2202_01284_gb300.render import DeviceScene, RenderSettings
    sc = S.shadow_scene(width=32, height=32, floor_bsdf=S.BSDF_BLEND)
    cam = sc.cameras[0]
    rng = np.random.default_rng(43)
    d = rng.normal(size=(sc.n_tris, 3, 3) if vertex else (sc.n_shapes, 3))
    st = RenderSettings(width=32, height=32, spp=6, max_depth=3, rr_depth=-1, seed=47)
    ds = DeviceScene(sc)
    _, dot = ds.jvp_reparam(st, dir_vertices=d, edge_spp=2) if vertex else ds.jvp_reparam(st, d, edge_spp=2)
    torch.cuda.synchronize()
    dot = dot[0].cpu().numpy().astype(np.float64)
    r = oracle_mod.render_in(cam, 6, 3, 47, -1, True)
    _, _, ref = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, vertex=vertex, dot_dir=d, edge_spp=2)
    c = cosine(dot.ravel(), ref.ravel())
    rel = np.abs(dot - ref).max() / np.abs(ref).max()
    print(f"random direction (vertex={vertex}): cosine {c:.7f} max rel {rel:.2e}")
    assert c >= 0.9999 and rel < 5e-3
