"""Pins of the oracle's reparameterized translation derivative (Sec. 4.7).

The estimator (warp field from auxiliary rays, Jacobian determinant, per-ray
log-derivative factors) is defined in oracle.cpp.  It is pinned here against
what the mathematics fixes independently of it:
  * the divergence on the sphere of analytic fields (closed forms);
  * the divergence of an actual warp field against central differences of the
    field itself (samples held fixed);
  * the expected derivative of a rendered image against closed forms (the
    projected area of a square seen against a uniform sky) and against central
    finite differences of the primal render, for moving occluders and lights.
The warp estimator is consistent, not unbiased: the tolerances below state the
bias measured at the default options (16 auxiliary rays).
"""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

pytestmark = pytest.mark.filterwarnings("ignore")


def test_sphere_divergence_closed_forms(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(20):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        e = rng.normal(size=3)
        # constant ambient field and its tangential part: div = -2 e.u; rotation: 0
        assert oracle_mod.sphere_div(0, u, e) == pytest.approx(-2 * e @ u, abs=1e-12)
        assert oracle_mod.sphere_div(1, u, e) == pytest.approx(0.0, abs=1e-12)
        assert oracle_mod.sphere_div(2, u, e) == pytest.approx(-2 * e @ u, abs=1e-12)


def _chart_coords(V, w, u, t):
    return (t @ V * (u @ w) - (t @ w) * (u @ V)) / (u @ w) ** 2


@pytest.mark.parametrize("param", [0, 2])
def test_warp_divergence_matches_finite_differences(oracle_mod, param):
    sc = S.occluder_sky()
    osc = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(4)
    o = np.zeros(3)
    n_checked = 0
    for trial in range(12):
        # directions near the square's right edge (x = 0.35 at depth 3)
        u = np.array([0.35 + rng.uniform(-0.05, 0.05), rng.uniform(-0.05, 0.25), -3.0])
        u /= np.linalg.norm(u)
        uni = rng.random(32)
        opts = dict(jackknife=0)
        V0, div, logd, n = oracle_mod.warp(osc, o, u, -1, uni, param, m=np.array([0.3, -0.2, 0.5]), **opts)
        if n == 0 or not np.any(V0):
            continue
        t1, t2 = oracle_mod.frame(u)
        h = 1e-5
        fd = 0.0
        for t in (t1, t2):
            vals = []
            for sgn in (1, -1):
                w = u + sgn * h * t
                w /= np.linalg.norm(w)
                V, _, _, _ = oracle_mod.warp(osc, o, u, -1, uni, param, at=w, **opts)
                vals.append(_chart_coords(V, w, u, t))
            fd += (vals[0] - vals[1]) / (2 * h)
        assert div == pytest.approx(fd, rel=1e-5, abs=1e-6 * max(1.0, abs(div)))
        # log-derivative = m . (tangential part of V) + div V
        vt = V0 - u * (u @ V0)
        assert logd == pytest.approx(np.array([0.3, -0.2, 0.5]) @ vt + div, rel=1e-9, abs=1e-12)
        n_checked += 1
    assert n_checked >= 6


def _sum_grad(oracle_mod, sc, spp, seed, **opts):
    cam = sc.cameras[0]
    r = oracle_mod.render_in(cam, spp, 2, seed, -1, True)
    g, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, np.ones((cam.height, cam.width, 3)), **opts)
    return g


def test_square_depth_and_lateral_closed_forms(oracle_mod):
    """A black square (side s, depth d) over a sky of radiance 1: the summed image
    is (image area - (s/d)^2) / pixel area per channel, so moving it toward the
    camera changes the sum by -2 s^2 / d^3 / pixel area per channel and moving it
    sideways not at all."""
    sc = S.occluder_sky(center=(0.15, 0.1), depth=3.0, side=0.4, width=64, height=64)
    th = np.tan(np.radians(20.0))
    pix_area = (2 * th / 64) ** 2
    exact_z = -3 * 2 * 0.4 ** 2 / 3.0 ** 3 / pix_area
    g = np.mean([_sum_grad(oracle_mod, sc, 256, seed)[0] for seed in (7, 8)], axis=0)
    print("square: reparameterized", g, "closed form z", exact_z)
    assert g[2] / exact_z == pytest.approx(1.0, abs=0.08)  # measured 0.96 (consistent estimator, N = 16)
    assert abs(g[0]) < 0.2 * abs(exact_z) and abs(g[1]) < 0.2 * abs(exact_z)
    # more auxiliary rays approach the closed form
    g32 = _sum_grad(oracle_mod, sc, 128, 9, n_aux=32)[0]
    assert abs(g32[2] / exact_z - 1.0) < 0.06


def test_shadow_scene_matches_finite_differences(oracle_mod):
    """Moving the light and the occluder of a lit floor, against central finite
    differences of the primal render (same random numbers on both sides of each
    difference; 1024 samples per pixel)."""
    sc = S.shadow_scene()
    cam = sc.cameras[0]
    g = _sum_grad(oracle_mod, sc, 64, 3)
    rf = oracle_mod.render_in(cam, 512, 2, 5, -1, True)
    h = 0.01
    fd = np.zeros((3, 3))
    for shape in (1, 2):
        for axis in range(3):
            off = np.zeros((3, 3))
            off[shape, axis] = h
            ip = oracle_mod.render(oracle_mod.OracleScene(sc.translated(off)), rf).sum()
            im = oracle_mod.render(oracle_mod.OracleScene(sc.translated(-off)), rf).sum()
            fd[shape, axis] = (ip - im) / (2 * h)
    print("reparameterized\n", g, "\nfinite differences\n", fd)
    for shape in (1, 2):
        scale = np.abs(fd[shape]).max()
        assert np.abs(g[shape] - fd[shape]).max() < 0.15 * scale
    # a plain (not reparameterized) derivative would be zero for every translation
    assert np.abs(g[1:]).max() > 0.5 * np.abs(fd[1:]).max()


@pytest.mark.parametrize("floor", [S.BSDF_DIFFUSE, S.BSDF_CONDUCTOR])
def test_vertex_gradients_sum_to_translation_gradients(oracle_mod, floor):
    """Moving every corner of a shape by the same vector is its translation: the
    per-corner gradients of a shape sum to its translation gradient (the normal
    terms, of the cosine and of a glossy BSDF value, cancel; the plane points'
    barycentric weights sum to one; the pixel-edge terms follow)."""
    sc = S.shadow_scene(width=32, height=32, floor_bsdf=floor)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], 8, 3, 21, -1, True)
    gi = np.random.default_rng(2).random((32, 32, 3)) + 0.5
    gt, _, _ = oracle_mod.grad_reparam(osc, r, gi)
    gv, _, _ = oracle_mod.grad_reparam(osc, r, gi, vertex=True)
    sums = np.zeros_like(gt)
    for t in range(sc.n_tris):
        sums[sc.tri_shape[t]] += gv[t].sum(axis=0)
    assert np.abs(sums - gt).max() <= 1e-9 * np.abs(gt).max()


def _corner_field(sc, shape, fn):
    """Per-corner displacement direction [n_tris, 3, 3]: fn(corner position) on `shape`."""
    v = np.zeros((sc.n_tris, 3, 3))
    for t in range(sc.n_tris):
        if sc.tri_shape[t] == shape:
            for k in range(3):
                v[t, k] = fn(sc.vertices[t, k].astype(np.float64))
    return v


def test_square_scaling_closed_form(oracle_mod):
    """Growing the square about its centre (corners move by eps (p - c)): its
    projected area grows by 2 (s/d)^2 per unit eps, a non-rigid motion."""
    sc = S.occluder_sky(center=(0.15, 0.1), depth=3.0, side=0.4, width=48, height=48)
    th = np.tan(np.radians(20.0))
    pix_area = (2 * th / 48) ** 2
    exact = -3 * 2 * (0.4 / 3.0) ** 2 / pix_area
    c = np.array([0.15, 0.1, -3.0])
    v = _corner_field(sc, 0, lambda p: p - c)
    r = oracle_mod.render_in(sc.cameras[0], 256, 2, 7, -1, True)
    gv, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, np.ones((48, 48, 3)), vertex=True)
    got = float((gv * v).sum())
    print("scaling: reparameterized", got, "closed form", exact)
    assert got / exact == pytest.approx(1.0, abs=0.1)


class _SquareCoverage:
    """Exact image of the black square over the uniform sky (radiance 1), seen
    face-on by the pinhole camera at the origin looking along -z: a pixel's value
    is 1 minus the area of its unit box covered by the square's projection, an
    axis-aligned rectangle in pixel coordinates (x right, y down)."""

    def __init__(self, w, h, side, vfov_deg=40.0):
        self.w, self.h, self.half = w, h, 0.5 * side
        self.th = np.tan(np.radians(0.5 * vfov_deg))

    def image(self, cx, cy, depth):
        k = 1.0 / (depth * self.th)
        x0, x1 = ((cx - self.half) * k + 1) * self.w / 2, ((cx + self.half) * k + 1) * self.w / 2
        y0, y1 = (1 - (cy + self.half) * k) * self.h / 2, (1 - (cy - self.half) * k) * self.h / 2
        i, j = np.arange(self.w), np.arange(self.h)
        ox = np.clip(np.minimum(i + 1, x1) - np.maximum(i, x0), 0, None)
        oy = np.clip(np.minimum(j + 1, y1) - np.maximum(j, y0), 0, None)
        return 1.0 - oy[:, None] * ox[None, :]

    def d_image(self, cx, cy, depth, axis, e=1e-6):
        """Derivative of the exact image along translation axis (z: toward the camera
        at z = 0 means depth decreases); the coverage is piecewise linear in the
        rectangle's sides, so a tiny central difference is exact to rounding."""
        d = np.zeros(3)
        d[axis] = e
        a = self.image(cx + d[0], cy + d[1], depth - d[2])
        b = self.image(cx - d[0], cy - d[1], depth + d[2])
        return (a - b) / (2 * e)


@pytest.mark.parametrize("axis", [0, 2])
def test_per_pixel_derivative_closed_form(oracle_mod, axis):
    """Per-pixel image derivative of a translated square against the exact one.  The
    warp keeps the square's silhouette fixed in the integration variable but moves
    each pixel's box, so only the interior terms plus the pixel-edge term give the
    per-pixel derivative: without the edge term the estimate is a blurred version
    whose relative error stays near 1 however many samples are taken."""
    cx, cy, depth, side, n = 0.15, 0.1, 3.0, 0.8, 32
    sq = _SquareCoverage(n, n, side)
    sc = S.occluder_sky(center=(cx, cy), depth=depth, side=side, width=n, height=n)
    osc = oracle_mod.OracleScene(sc)
    exact = sq.d_image(cx, cy, depth, axis)

    def rel_err(spp, edge_spp):
        r = oracle_mod.render_in(sc.cameras[0], spp, 4, 5, -1, True)
        _, img, dot = oracle_mod.grad_reparam(osc, r, dot_param=axis, edge_spp=edge_spp)
        assert np.abs(img[..., 0] - sq.image(cx, cy, depth)).max() < 0.25
        return np.linalg.norm(dot[..., 0] - exact) / np.linalg.norm(exact)

    e = rel_err(1024, 256)
    e0 = rel_err(256, 0)
    print("per-pixel relative L2 error with / without the edge term", e, e0)
    assert e < 0.15  # measured 0.10 / 0.09 (sampling noise plus the N = 16 warp bias)
    assert e0 > 0.9


def test_per_pixel_scaling_derivative_closed_form(oracle_mod):
    """Vertex mode with a non-rigid motion: the square grows about its centre
    (corner velocities p - c, the image derivative along that direction of all
    corner coordinates); per pixel against the exact derivative of the coverage
    image with respect to the side, times the side."""
    cx, cy, depth, side, n = 0.15, 0.1, 3.0, 0.8, 32
    sc = S.occluder_sky(center=(cx, cy), depth=depth, side=side, width=n, height=n)
    c = np.array([cx, cy, -depth])
    v = _corner_field(sc, 0, lambda p: p - c)
    e = 1e-6
    exact = side * (_SquareCoverage(n, n, side + e).image(cx, cy, depth)
                    - _SquareCoverage(n, n, side - e).image(cx, cy, depth)) / (2 * e)
    r = oracle_mod.render_in(sc.cameras[0], 1024, 4, 5, -1, True)
    _, _, dot = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, vertex=True, dot_dir=v, edge_spp=256)
    err = np.linalg.norm(dot[..., 0] - exact) / np.linalg.norm(exact)
    print("scaling, per-pixel relative L2 error", err, "summed", dot[..., 0].sum(), exact.sum())
    assert err < 0.15


def test_per_pixel_derivative_across_the_image_border(oracle_mod):
    """A square that crosses the right image border and moves in depth: its edges
    slide through the image border, so the border pixels change by the flux through
    their outer edges.  Without a window the image-border edges carry that flux and
    the per-pixel derivative matches the exact one; the optional 4-pixel window
    (warp taken to 0 at the border) biases it."""
    cx, cy, depth, side, n = 1.25, 0.1, 3.0, 0.8, 32
    sq = _SquareCoverage(n, n, side)
    sc = S.occluder_sky(center=(cx, cy), depth=depth, side=side, width=n, height=n)
    osc = oracle_mod.OracleScene(sc)
    exact = sq.d_image(cx, cy, depth, 2)
    r = oracle_mod.render_in(sc.cameras[0], 1024, 4, 5, -1, True)
    errs = {}
    for border in (0.0, 4.0):
        _, _, dot = oracle_mod.grad_reparam(osc, r, dot_param=2, edge_spp=256, border=border)
        errs[border] = np.linalg.norm(dot[..., 0] - exact) / np.linalg.norm(exact)
    print("per-pixel relative L2 error, no window / 4-pixel window:", errs)
    assert errs[0.0] < 0.15  # measured 0.10
    assert errs[4.0] > 0.2   # measured 0.25


@pytest.mark.parametrize("vertex", [False, True])
def test_reparameterization_is_the_identity_in_the_primal(oracle_mod, vertex):
    """Sec. 4.7: a reparameterized ray returns the same direction in the primal, so
    the image that comes with the reparameterized derivative is the plain render of
    the same samples, exactly (its auxiliary rays draw from their own streams)."""
    sc = S.shadow_scene(width=20, height=20, floor_bsdf=S.BSDF_BLEND)
    r = oracle_mod.render_in(sc.cameras[0], 4, 4, 13, 2, True)
    osc = oracle_mod.OracleScene(sc)
    _, img, _ = oracle_mod.grad_reparam(osc, r, np.ones((20, 20, 3)), vertex=vertex)
    np.testing.assert_array_equal(img, oracle_mod.render(osc, r))


def test_moving_the_camera_is_moving_the_scene_the_other_way(oracle_mod):
    """The identity behind the camera-translation gradient: with nothing at infinity
    but a uniform (or no) environment, a render from a camera moved by d equals the
    render of every shape moved by -d, sample for sample."""
    sc = S.shadow_scene(width=24, height=24)
    d = np.array([0.05, -0.03, 0.08])
    a = oracle_mod.render(oracle_mod.OracleScene(sc), oracle_mod.render_in(sc.camera_moved(d).cameras[0], 8, 3, 11,
                                                                             -1, True))
    moved = sc.translated(-np.tile(d, (sc.n_shapes, 1)))
    b = oracle_mod.render(oracle_mod.OracleScene(moved), oracle_mod.render_in(sc.cameras[0], 8, 3, 11, -1, True))
    diff = np.abs(a - b)
    print("camera vs scene motion: max diff", diff.max(), "pixels differing by > 1e-6:", int((diff > 1e-6).sum()))
    # equal up to the float32 rounding of the moved vertices (measured 1.7e-8); a
    # decision flipping at an edge would show as a few pixels far off
    assert (diff > 1e-6).mean() < 0.01
    assert np.median(diff) < 1e-7


def test_camera_translation_matches_finite_differences(oracle_mod):
    """Moving the camera is moving every shape the opposite way (nothing lies at a
    finite distance outside the scene): minus the sum of all shapes' translation
    gradients against central finite differences of renders from moved cameras.
    Everything in view slides, so the flux through the image border (the
    image-border edges of the pixel-edge term) is most of it; the scene is
    symmetric in z, so that component vanishes."""
    import dataclasses
    sc = S.shadow_scene(width=48, height=48)
    cam = sc.cameras[0]
    osc = oracle_mod.OracleScene(sc)
    ones = np.ones((48, 48, 3))
    r = oracle_mod.render_in(cam, 64, 3, 3, -1, True)
    g, _, _ = oracle_mod.grad_reparam(osc, r, ones, edge_spp=64)
    g_int, _, _ = oracle_mod.grad_reparam(osc, r, ones, edge_spp=0)
    got, got_int = -g.sum(axis=0), -g_int.sum(axis=0)
    fd = np.zeros(3)
    h = 0.01
    for a in range(3):
        off = np.zeros(3)
        off[a] = h
        img = [oracle_mod.render(osc, oracle_mod.render_in(
            dataclasses.replace(cam, origin=tuple(np.add(cam.origin, sg * off)),
                                target=tuple(np.add(cam.target, sg * off))), 1024, 3, 5, -1, True))
            for sg in (1, -1)]
        fd[a] = (img[0].sum() - img[1].sum()) / (2 * h)
    print("camera translation: reparameterized", got, "interior terms only", got_int, "finite differences", fd)
    scale = np.abs(fd).max()
    assert np.abs(got[:2] - fd[:2]).max() < 0.1 * scale   # measured 2 % / 4 %
    assert abs(got[2]) < 0.2 * scale
    assert np.abs(got_int[:2] - fd[:2]).max() > scale     # the border flux is needed


def test_sharp_loss_gradient_closed_form(oracle_mod):
    """Gradient of the unblurred per-pixel L2 loss against a shifted target, the
    case the pixel-edge term exists for: against the exact value from the coverage
    image, per axis."""
    cx, cy, depth, side, n = 0.15, 0.1, 3.0, 0.8, 32
    sq = _SquareCoverage(n, n, side)
    sc = S.occluder_sky(center=(cx, cy), depth=depth, side=side, width=n, height=n)
    img = sq.image(cx, cy, depth)
    gi = np.repeat((2.0 * (img - sq.image(cx + 0.03, cy - 0.02, depth - 0.1)))[..., None], 3, axis=2)
    exact = np.array([3.0 * (gi[..., 0] * sq.d_image(cx, cy, depth, a)).sum() for a in range(3)])
    r = oracle_mod.render_in(sc.cameras[0], 256, 4, 5, -1, True)
    g, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, gi, edge_spp=16)
    g0, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, gi, edge_spp=0)
    print("sharp loss: with edges", g[0], "without", g0[0], "exact", exact)
    np.testing.assert_allclose(g[0], exact, rtol=0.12)  # measured 5 %, 9 %, 6 %
    assert abs(g0[0, 0] / exact[0]) < 0.5  # interior terms alone: 0.28 of it


@pytest.mark.parametrize("bsdf", [S.BSDF_CONDUCTOR, S.BSDF_BLEND, S.BSDF_DIFFUSE])
def test_bsdf_normal_derivative_matches_finite_differences(oracle_mod, bsdf):
    """Vertex mode turns a triangle's normal, and a glossy BSDF value depends on it.
    The oracle's dual-number derivative of log f_c with respect to each corner
    coordinate against central differences of log f evaluated through another
    orthonormal frame (Gram-Schmidt) of the perturbed normal; 0 for diffuse."""
    rng = np.random.default_rng(17)
    params = oracle_mod.bsdf_params(albedo=(0.6, 0.4, 0.3), alpha=0.25, f0=(0.9, 0.6, 0.3), wd=0.5)
    for trial in range(4):
        v = rng.normal(size=(3, 3))
        c = np.cross(v[1] - v[0], v[2] - v[0])
        n = c / np.linalg.norm(c) * (1 if trial % 2 else -1)
        def unit_above(k):
            while True:
                w = rng.normal(size=3)
                w /= np.linalg.norm(w)
                if w @ n > 0.2:
                    return w
        wi, wo = unit_above(0), unit_above(1)

        def log_f(vv):
            cc = np.cross(vv[1] - vv[0], vv[2] - vv[0])
            nn = cc / np.linalg.norm(cc) * np.sign(cc @ n)
            s = np.array([1.0, 0.3, -0.2])
            s = s - nn * (s @ nn)
            s /= np.linalg.norm(s)
            t = np.cross(nn, s)
            loc = lambda w: np.array([w @ s, w @ t, w @ nn])
            return np.log(oracle_mod.bsdf_eval(bsdf, params, loc(wi), loc(wo))[0])

        got = oracle_mod.bsdf_normal_dlog(bsdf, params, v, n, wi, wo)
        h = 1e-6
        for k in range(3):
            for a in range(3):
                vp, vm = v.copy(), v.copy()
                vp[k, a] += h
                vm[k, a] -= h
                fd = (log_f(vp) - log_f(vm)) / (2 * h)
                np.testing.assert_allclose(got[k, a], fd, rtol=1e-5, atol=1e-6)
        if bsdf == S.BSDF_DIFFUSE:
            assert not got.any()
        else:
            assert np.abs(got).max() > 1e-2


def _rotation_field(center, axis, sc, shape):
    a = np.asarray(axis, np.float64)
    a /= np.linalg.norm(a)
    return _corner_field(sc, shape, lambda p: np.cross(a, p - np.asarray(center)))


def test_tilting_light_and_occluder_match_finite_differences(oracle_mod):
    """Tilting the light or the occluder (corners rotate about the centre, which turns
    their normals) against central finite differences of the primal render."""
    sc = S.shadow_scene(width=48, height=48)
    cam = sc.cameras[0]
    r = oracle_mod.render_in(cam, 32, 2, 3, -1, True)
    gv, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, np.ones((48, 48, 3)), vertex=True)
    rf = oracle_mod.render_in(cam, 512, 2, 5, -1, True)
    for shape, center, axis in ((1, (-1.2, 2.0, 0.0), (0, 0, 1)), (1, (-1.2, 2.0, 0.0), (1, 0, 0)),
                                (2, (-0.6, 0.8, 0.0), (0, 0, 1)), (2, (-0.6, 0.8, 0.0), (1, 0, 0))):
        v = _rotation_field(center, axis, sc, shape)
        got = float((gv * v).sum())
        h = 0.02
        vals = []
        for sgn in (1, -1):
            moved = sc.translated(np.zeros((3, 3)))
            moved.vertices = (sc.vertices.astype(np.float64) + sgn * h * v).astype(np.float32)
            vals.append(oracle_mod.render(oracle_mod.OracleScene(moved), rf).sum())
        fd = (vals[0] - vals[1]) / (2 * h)
        print(f"tilt shape {shape} axis {axis}: reparameterized {got:.2f} finite differences {fd:.2f}")
        assert abs(got - fd) < 0.15 * abs(fd) + 5.0


@pytest.mark.parametrize("bsdf,tol", [(S.BSDF_CONDUCTOR, 0.1), (S.BSDF_BLEND, 0.1)])
def test_tilting_glossy_floor_matches_finite_differences(oracle_mod, bsdf, tol):
    """Tilting the glossy floor under the light (its corners rotate about the z axis):
    the highlight follows the turning normal through the BSDF value, a term of the
    vertex-position derivative that a translation does not have.  Against central
    finite differences of the primal render (measured 2.4 % / 1.8 % off; 6 % / 14 %
    with the optional border window, whose band the floor crosses; without the BSDF's
    normal term the conductor's derivative has the wrong sign)."""
    sc = S.shadow_scene(width=48, height=48, floor_bsdf=bsdf, floor_alpha=0.3)
    cam = sc.cameras[0]
    r = oracle_mod.render_in(cam, 64, 2, 3, -1, True)
    gv, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, np.ones((48, 48, 3)), vertex=True)
    v = _rotation_field((0.0, 0.0, 0.0), (0, 0, 1), sc, 0)
    got = float((gv * v).sum())
    rf = oracle_mod.render_in(cam, 1024, 2, 5, -1, True)
    h = 0.005
    vals = []
    for sgn in (1, -1):
        moved = sc.translated(np.zeros((3, 3)))
        moved.vertices = (sc.vertices.astype(np.float64) + sgn * h * v).astype(np.float32)
        vals.append(oracle_mod.render(oracle_mod.OracleScene(moved), rf).sum())
    fd = (vals[0] - vals[1]) / (2 * h)
    print(f"glossy floor tilt: reparameterized {got:.1f} finite differences {fd:.1f}")
    assert abs(got - fd) < tol * abs(fd)


@pytest.mark.parametrize("bsdf", [S.BSDF_CONDUCTOR, S.BSDF_BLEND])
def test_glossy_receiver_matches_finite_differences(oracle_mod, bsdf):
    """A glossy floor (GGX conductor, or the diffuse + GGX blend): its BSDF value
    depends on both directions, so a ray's warp also turns the next vertex's
    incident direction.  Moving the light and the occluder against central finite
    differences of the primal render."""
    sc = S.shadow_scene(width=48, height=48, floor_bsdf=bsdf, floor_alpha=0.3)
    cam = sc.cameras[0]
    r = oracle_mod.render_in(cam, 64, 2, 3, -1, True)
    g, _, _ = oracle_mod.grad_reparam(oracle_mod.OracleScene(sc), r, np.ones((48, 48, 3)))
    rf = oracle_mod.render_in(cam, 1024, 2, 5, -1, True)
    h = 0.01
    fd = np.zeros((3, 3))
    for shape in (1, 2):
        for axis in range(3):
            off = np.zeros((3, 3))
            off[shape, axis] = h
            ip = oracle_mod.render(oracle_mod.OracleScene(sc.translated(off)), rf).sum()
            im = oracle_mod.render(oracle_mod.OracleScene(sc.translated(-off)), rf).sum()
            fd[shape, axis] = (ip - im) / (2 * h)
    print("reparameterized\n", g, "\nfinite differences\n", fd)
    for shape in (1, 2):
        assert np.abs(g[shape] - fd[shape]).max() < 0.25 * np.abs(fd[shape]).max()


@pytest.mark.parametrize("kappa", [2.0, 50.0, 1000.0])
def test_vmf_sampler_matches_the_distribution(oracle_mod, kappa):
    """Auxiliary directions follow the von Mises-Fisher law p(w) ~ exp(kappa w.z):
    cos(theta) has CDF (e^{kappa c} - e^{-kappa}) / (e^{kappa} - e^{-kappa}) and the
    azimuth is uniform; the directions are unit vectors."""
    rng = np.random.default_rng(int(kappa))
    u = rng.random((20000, 2))
    w = np.array([oracle_mod.vmf(a, b, kappa) for a, b in u])
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0, atol=1e-12)
    c = np.sort(w[:, 2])
    emp = np.arange(1, len(c) + 1) / len(c)
    cdf = (np.exp(kappa * (c - 1.0)) - np.exp(-2 * kappa)) / (1.0 - np.exp(-2 * kappa))
    assert np.abs(emp - cdf).max() < 0.015          # Kolmogorov-Smirnov distance
    phi = np.arctan2(w[:, 1], w[:, 0])
    hist, _ = np.histogram(phi, bins=8, range=(-np.pi, np.pi))
    assert np.abs(hist / len(phi) - 1 / 8).max() < 0.01
    # mean cosine: coth(kappa) - 1/kappa
    assert w[:, 2].mean() == pytest.approx(1 / np.tanh(kappa) - 1 / kappa, abs=3 / np.sqrt(len(c)) * w[:, 2].std() + 1e-9)
