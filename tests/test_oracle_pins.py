"""Pins of the FP64 oracle against facts fixed outside of it (CPU only).

Each test checks one part of the oracle against a published test vector, a
closed form, an invariant, brute force, or finite differences -- never against
a retyped copy of its own formula.
"""
import math
import os

import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- RNG
def test_pcg32_reference_vector(oracle_mod):
    """O'Neill's published pcg32-demo outputs for (initstate 42, initseq 54)."""
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "pcg32_demo.txt")) if l.strip() and not l.startswith("#")]
    st = int(lines[0].split()[1])
    sq = int(lines[1].split()[1])
    want = [int(x, 16) for x in lines[2:]]
    got = oracle_mod.pcg32(st, sq, len(want))
    assert [int(x) for x in got] == want


# ---------------------------------------------------------------- frames and samplers
def test_frame_is_orthonormal_right_handed(oracle_mod):
    rng = np.random.default_rng(1)
    ns = rng.normal(size=(200, 3))
    ns /= np.linalg.norm(ns, axis=1, keepdims=True)
    ns = np.concatenate([ns, np.eye(3), -np.eye(3)])
    for n in ns:
        s, t = oracle_mod.frame(n)
        M = np.stack([s, t, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(s, t), n, atol=1e-12)


def _hemisphere_grid(n_theta=200, n_phi=400):
    th = (np.arange(n_theta) + 0.5) / n_theta * (np.pi / 2)
    ph = (np.arange(n_phi) + 0.5) / n_phi * 2 * np.pi
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    dw = (np.sin(T) * (np.pi / 2 / n_theta) * (2 * np.pi / n_phi)).reshape(-1)
    return d, dw


def test_cosine_sampler_moments(oracle_mod):
    """Cosine-weighted hemisphere (Sec. 3.1 example): E[cos] = 2/3, E[cos^2] = 1/2, E[x] = E[y] = 0."""
    rng = np.random.default_rng(2)
    p = oracle_mod.bsdf_params()
    u = rng.random((20000, 2))
    wo = np.array([oracle_mod.bsdf_sample(S.BSDF_DIFFUSE, p, [0, 0, 1], 0.0, a, b)[1] for a, b in u])
    assert np.allclose(np.linalg.norm(wo, axis=1), 1.0, atol=1e-12)
    se = 1.0 / math.sqrt(len(u))
    assert abs(wo[:, 2].mean() - 2 / 3) < 4 * se
    assert abs((wo[:, 2] ** 2).mean() - 0.5) < 4 * se
    assert abs(wo[:, 0].mean()) < 4 * se and abs(wo[:, 1].mean()) < 4 * se


@pytest.mark.parametrize("bsdf", [S.BSDF_DIFFUSE, S.BSDF_CONDUCTOR, S.BSDF_BLEND])
def test_bsdf_pdf_normalised_and_energy(oracle_mod, bsdf):
    """Quadrature over the hemisphere: pdf integrates to the sampler's success rate; albedo <= 1."""
    d, dw = _hemisphere_grid()
    p = oracle_mod.bsdf_params(albedo=(0.7, 0.5, 0.3), alpha=0.35, f0=(0.9, 0.6, 0.3))
    wi = np.array([0.3, -0.2, 0.0])
    wi[2] = math.sqrt(1 - wi[0] ** 2 - wi[1] ** 2)
    pdf_int = 0.0
    alb = np.zeros(3)
    for w, a in zip(d, dw):
        f, pdf = oracle_mod.bsdf_eval(bsdf, p, wi, w)
        pdf_int += pdf * a
        alb += f * w[2] * a
    if bsdf == S.BSDF_DIFFUSE:
        assert abs(pdf_int - 1.0) < 1e-3
        assert np.allclose(alb, [0.7, 0.5, 0.3], atol=2e-3)
    else:
        rng = np.random.default_rng(3)
        ok = np.mean([oracle_mod.bsdf_sample(bsdf, p, wi, *rng.random(3))[0] for _ in range(20000)])
        assert abs(pdf_int - ok) < 0.01
        assert np.all(alb <= 1.0 + 1e-3)


def test_ggx_sampler_matches_pdf(oracle_mod):
    """Histogram of sampled cos(theta_o) vs the integral of the pdf over each bin."""
    p = oracle_mod.bsdf_params(alpha=0.3)
    wi = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(4)
    cos = []
    for _ in range(40000):
        ok, wo = oracle_mod.bsdf_sample(S.BSDF_CONDUCTOR, p, wi, *rng.random(3))
        if ok:
            cos.append(wo[2])
    cos = np.array(cos)
    edges = np.linspace(0, 1, 11)
    hist = np.histogram(cos, edges)[0] / 40000
    d, dw = _hemisphere_grid(400, 8)
    pdf = np.array([oracle_mod.bsdf_eval(S.BSDF_CONDUCTOR, p, wi, w)[1] for w in d])
    want = np.array([np.sum((pdf * dw)[(d[:, 2] >= a) & (d[:, 2] < b)]) for a, b in zip(edges[:-1], edges[1:])])
    assert np.all(np.abs(hist - want) < 5 * np.sqrt(want / 40000) + 2e-3)


@pytest.mark.parametrize("bsdf", [S.BSDF_DIFFUSE, S.BSDF_CONDUCTOR, S.BSDF_BLEND])
def test_bsdf_reciprocity(oracle_mod, bsdf):
    rng = np.random.default_rng(5)
    p = oracle_mod.bsdf_params(albedo=(0.6, 0.4, 0.2), alpha=0.25, f0=(0.9, 0.5, 0.1))
    for _ in range(100):
        a, b = rng.normal(size=(2, 3))
        a[2], b[2] = abs(a[2]), abs(b[2])
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        fa, _ = oracle_mod.bsdf_eval(bsdf, p, a, b)
        fb, _ = oracle_mod.bsdf_eval(bsdf, p, b, a)
        assert np.allclose(fa, fb, rtol=1e-12, atol=0)


def test_ggx_small_alpha_is_mirror(oracle_mod):
    p = oracle_mod.bsdf_params(alpha=1e-4)
    wi = np.array([0.4, 0.1, 0.0])
    wi[2] = math.sqrt(1 - 0.17)
    for u in [(0.1, 0.2, 0.9), (0.5, 0.7, 0.3)]:
        ok, wo = oracle_mod.bsdf_sample(S.BSDF_CONDUCTOR, p, wi, *u)
        assert ok and np.allclose(wo, [-wi[0], -wi[1], wi[2]], atol=1e-3)


def test_fresnel_textbook_values(oracle_mod):
    eta = 1.5
    assert abs(oracle_mod.fresnel(1.0, eta) - ((eta - 1) / (eta + 1)) ** 2) < 1e-15   # normal incidence: 0.04
    assert oracle_mod.fresnel(0.0, eta) == 1.0                                        # grazing
    th_b = math.atan(eta)                                                             # Brewster: R_p = 0
    ci = math.cos(th_b)
    ct = math.sqrt(1 - (1 - ci * ci) / eta ** 2)
    rs = ((ci - eta * ct) / (ci + eta * ct)) ** 2
    assert abs(oracle_mod.fresnel(ci, eta) - rs / 2) < 1e-15
    crit = math.sqrt(1 - (1 / eta) ** 2)                                              # from inside: TIR
    assert oracle_mod.fresnel(crit * 0.999, 1 / eta) == 1.0
    assert oracle_mod.fresnel(crit * 1.01, 1 / eta) < 1.0


def test_dfactors_match_finite_differences(oracle_mod):
    """Analytic (df/dtheta)/f used by the tape vs central differences of the BSDF value."""
    rng = np.random.default_rng(6)
    for bsdf in (S.BSDF_DIFFUSE, S.BSDF_CONDUCTOR, S.BSDF_BLEND):
        for _ in range(20):
            a, b = rng.normal(size=(2, 3))
            a[2], b[2] = abs(a[2]) + 0.05, abs(b[2]) + 0.05
            a /= np.linalg.norm(a)
            b /= np.linalg.norm(b)
            alb = rng.uniform(0.2, 0.8, 3)
            alpha = rng.uniform(0.1, 0.5)
            p = oracle_mod.bsdf_params(albedo=alb, alpha=alpha, f0=(0.04, 0.04, 0.04))
            f, _ = oracle_mod.bsdf_eval(bsdf, p, a, b)
            d_alb, d_alpha = oracle_mod.bsdf_dfactors(bsdf, p, a, b)
            h = 1e-6
            for c in range(3):
                pp, pm = p.copy(), p.copy()
                pp[c] += h
                pm[c] -= h
                fd = (oracle_mod.bsdf_eval(bsdf, pp, a, b)[0][c] - oracle_mod.bsdf_eval(bsdf, pm, a, b)[0][c]) / (2 * h)
                assert abs(fd / f[c] - d_alb[c]) < 1e-6 * max(1, abs(d_alb[c]))
            pp, pm = p.copy(), p.copy()
            pp[3] += h
            pm[3] -= h
            fd = (oracle_mod.bsdf_eval(bsdf, pp, a, b)[0] - oracle_mod.bsdf_eval(bsdf, pm, a, b)[0]) / (2 * h)
            assert np.allclose(fd / f, d_alpha, rtol=1e-5, atol=1e-6)


# ---------------------------------------------------------------- traversal
def test_bvh_matches_brute_force(oracle_mod):
    rng = np.random.default_rng(7)
    sc = S.cornell()
    # plus a random soup of 600 triangles
    soup = rng.uniform(-1, 1, size=(600, 3, 3)).astype(np.float32)
    soup = soup[:, :1] + 0.2 * (soup - soup[:, :1])
    for scene in (sc, sc.__class__(**{**sc.__dict__, "vertices": soup, "uvs": np.zeros((600, 3, 2), np.float32),
                                      "tri_shape": np.zeros(600, np.int32)})):
        osc = oracle_mod.OracleScene(scene)
        o = rng.uniform(-0.9, 0.9, size=(3000, 3)) + np.array([0, 1.0 if scene is sc else 0, 0])
        d = rng.normal(size=(3000, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        t1, p1 = oracle_mod.trace(osc, o, d, brute=False)
        t2, p2 = oracle_mod.trace(osc, o, d, brute=True)
        assert np.array_equal(p1, p2)
        assert np.array_equal(t1, t2)


# ---------------------------------------------------------------- closed forms of the integrator
@pytest.mark.parametrize("a,D", [(0.5, 5), (0.8, 3), (0.3, 8)])
def test_white_furnace_bsdf_only_is_exact(oracle_mod, a, D):
    """Closed enclosure, Le = E everywhere, albedo a, BSDF sampling only:
    every sample equals E * sum_{k<D} a^k (the cosine-sampling weight is a)."""
    E = 1.0
    sc = S.furnace(a, E, 8, 8)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], spp=4, max_depth=D, seed=11, nee=False)
    img, sl, _ = oracle_mod.render(osc, r, per_sample=True)
    a32 = float(np.float32(a))
    want = E * sum(a32 ** k for k in range(D))
    assert np.allclose(sl, want, rtol=1e-12)


def test_white_furnace_nee_mis_unbiased(oracle_mod):
    a, E, D = 0.5, 1.0, 6
    sc = S.furnace(a, E, 16, 16)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], spp=16, max_depth=D, seed=12, nee=True)
    _, sl, _ = oracle_mod.render(osc, r, per_sample=True)
    x = sl[..., 0].ravel()
    want = E * (1 - a ** D) / (1 - a)
    assert abs(x.mean() - want) < 4 * x.std() / math.sqrt(x.size)


def test_lit_plane(oracle_mod):
    """Diffuse plane (albedo a) under uniform env L: radiance a*L; exact without light sampling."""
    a, L = 0.6, 1.5
    sc = S.lit_plane(a, L)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], spp=4, max_depth=3, seed=13, nee=False)
    _, sl, _ = oracle_mod.render(osc, r, per_sample=True)
    want = float(np.float32(a)) * L
    assert np.allclose(sl, want, rtol=1e-12)
    r = oracle_mod.render_in(sc.cameras[0], spp=32, max_depth=3, seed=13, nee=True)
    _, sl, _ = oracle_mod.render(osc, r, per_sample=True)
    x = sl[..., 1].ravel()
    assert abs(x.mean() - want) < 4 * x.std() / math.sqrt(x.size)


def test_env_pdf_integrates_to_one(oracle_mod):
    sc = S.spheres(n_spheres=1, level=0, ground_quads=1, tex_res=16, env_size=(128, 64))
    osc = oracle_mod.OracleScene(sc)
    n_t, n_p = 256, 512
    th = (np.arange(n_t) + 0.5) / n_t * np.pi
    ph = (np.arange(n_p) + 0.5) / n_p * 2 * np.pi
    tot = 0.0
    for t in th:
        for p in ph[::4]:
            d = [math.sin(t) * math.cos(p), math.cos(t), math.sin(t) * math.sin(p)]
            tot += oracle_mod.env_pdf(osc, d) * math.sin(t) * (np.pi / n_t) * (2 * np.pi / n_p) * 4
    assert abs(tot - 1.0) < 1e-2


def test_env_importance_sampling_unbiased(oracle_mod):
    """Non-uniform sky with a sun: light sampling + MIS and BSDF-only sampling agree in expectation."""
    sc = S.lit_plane(0.5, 1.0, env_size=(64, 32))
    sc.env = S.sky_env(64, 32, sun_radius_deg=4.0, sun_radiance=50.0)
    osc = oracle_mod.OracleScene(sc)
    outs = []
    for nee, spp in ((True, 64), (False, 256)):
        r = oracle_mod.render_in(sc.cameras[0], spp=spp, max_depth=2, seed=17, nee=nee)
        _, sl, _ = oracle_mod.render(osc, r, per_sample=True)
        x = sl[..., 0].ravel()
        outs.append((x.mean(), x.std() / math.sqrt(x.size)))
    (m1, s1), (m2, s2) = outs
    assert abs(m1 - m2) < 4 * math.hypot(s1, s2)


# ---------------------------------------------------------------- gradients
def _cornell_grad_setup(oracle_mod, spp=4):
    sc = S.cornell(width=32, height=32)
    cam = sc.cameras[0]
    tgt = sc.with_params(albedo=S.cornell_target_albedo(sc.albedo))
    T = oracle_mod.render(oracle_mod.OracleScene(tgt), oracle_mod.render_in(cam, 8, 4, seed=99))
    r = oracle_mod.render_in(cam, spp, 4, seed=7)
    return sc, T, r


def test_albedo_gradient_tape_dual_fd(oracle_mod):
    """The image is polynomial in the albedos and sampling does not depend on them, so the
    Richardson-extrapolated central difference of the fixed-seed loss is exact to ~1e-9."""
    sc, T, r = _cornell_grad_setup(oracle_mod)

    def loss(alb):
        I = oracle_mod.render(oracle_mod.OracleScene(sc.with_params(albedo=alb)), r)
        return np.mean((I - T) ** 2), I
    _, I = loss(sc.albedo)
    gi = 2 * (I - T) / I.size
    ga, _, _ = oracle_mod.grad_tape(oracle_mod.OracleScene(sc), r, gi)
    gd = oracle_mod.grad_dual(oracle_mod.OracleScene(sc), r, gi, [(0, a, c, 0) for a in range(5) for c in range(3)])
    assert np.allclose(ga.ravel(), gd, rtol=1e-10, atol=1e-18)

    def cd(a, c, h):
        ap, am = sc.albedo.copy(), sc.albedo.copy()
        ap[a, c] += h
        am[a, c] -= h
        return (loss(ap)[0] - loss(am)[0]) / (np.float64(ap[a, c]) - np.float64(am[a, c]))
    scale = np.abs(gd).max()
    for a, c in [(0, 0), (1, 1), (2, 2), (3, 0), (4, 1)]:
        h = 2.0 ** -9
        rich = (4 * cd(a, c, h / 2) - cd(a, c, h)) / 3
        assert abs(rich - ga[a, c]) < 1e-7 * scale


def test_texel_and_roughness_gradients(oracle_mod):
    """Texels: FD exact (texels enter linearly, sampling independent of them).
    Roughness: sampling depends on alpha, so the detached derivative is pinned by
    tape == dual (two independent derivative engines) rather than by FD."""
    sc = S.cornell96(width=24, height=24, tex_res=256)
    cam = sc.cameras[0]
    r = oracle_mod.render_in(cam, 2, 4, seed=5)
    tgt = sc.with_params(textures=[S.cornell96_target_texture(sc.textures[0])])
    T = oracle_mod.render(oracle_mod.OracleScene(tgt), oracle_mod.render_in(cam, 4, 4, seed=6))
    osc = oracle_mod.OracleScene(sc)
    I = oracle_mod.render(osc, r)
    gi = 2 * (I - T) / I.size
    _, gt, gr = oracle_mod.grad_tape(osc, r, gi)
    g = gt[0]
    # texels with the largest gradients + roughness entries
    flat = np.abs(g[..., :3]).reshape(-1)
    top = np.argsort(flat)[-6:]
    sel = [(1, 0, int(i // 3), int(i % 3)) for i in top] + [(2, k, 0, 0) for k in np.argsort(np.abs(gr))[-4:]]
    gd = oracle_mod.grad_dual(osc, r, gi, sel)
    want = np.array([g.reshape(-1, 4)[b, c] for (_, _, b, c) in sel[:6]] + [gr[k] for (_, k, _, _) in sel[6:]])
    assert np.allclose(gd, want, rtol=1e-9, atol=1e-15)
    tex = sc.textures[0]
    for (_, _, b, c) in sel[:3]:
        y, x = divmod(b, tex.shape[1])
        vals = []
        for h in (2.0 ** -8, 2.0 ** -9):
            tp, tm = tex.copy(), tex.copy()
            tp[y, x, c] += h
            tm[y, x, c] -= h
            Lp = np.mean((oracle_mod.render(oracle_mod.OracleScene(sc.with_params(textures=[tp])), r) - T) ** 2)
            Lm = np.mean((oracle_mod.render(oracle_mod.OracleScene(sc.with_params(textures=[tm])), r) - T) ** 2)
            vals.append((Lp - Lm) / (np.float64(tp[y, x, c]) - np.float64(tm[y, x, c])))
        rich = (4 * vals[1] - vals[0]) / 3
        assert abs(rich - g[y, x, c]) < 1e-7 * np.abs(flat).max()


@pytest.mark.parametrize("x,n,a", [(1.7, 0, 0.5), (1.7, 1, 2.0), (-0.8, 5, 3.0), (2.5, 9, 0.1)])
def test_dual_numbers_on_the_toy_programs(oracle_mod, x, n, a):
    """The paper's AD toys (Fig. 1, x^n by repeated multiplication; Fig. 6, the
    exponential density a exp(-a x) with x detached) through the oracle's dual
    numbers, against their closed-form derivatives n x^(n-1) and
    exp(-a x)(1 - a x)."""
    y, dy, e, de = oracle_mod.dual_toys(x, n, a)
    assert y == pytest.approx(x ** n, rel=1e-14)
    assert dy == pytest.approx(n * x ** (n - 1) if n else 0.0, rel=1e-13, abs=1e-15)
    assert e == pytest.approx(a * np.exp(-a * x), rel=1e-14)
    assert de == pytest.approx(np.exp(-a * x) * (1.0 - a * x), rel=1e-13)
