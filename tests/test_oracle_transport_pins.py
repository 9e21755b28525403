"""Pins of the oracle's dielectric transport, Russian roulette, GGX masking term
and radiance-cache training targets (CPU only).

Each part is checked against physics or mathematics fixed outside the oracle:
Snell's law and the mirror law, the invariance of L / n^2 through a lossless
interface (a glass sphere in a uniform sky), the unbiasedness of roulette in a
closed-form furnace together with the empirical continuation frequencies,
Heitz's weak white furnace for the Smith masking function of GGX (Heitz 2014,
"Understanding the masking-shadowing function in microfacet-based BRDFs"), and
the zero-variance outgoing radiance of the white furnace for the training
targets.
"""
import math

import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------- dielectric event
@pytest.mark.parametrize("eta", [1.5, 1.33])
def test_dielectric_snell_mirror_and_weights(oracle_mod, eta):
    """Refraction obeys sin(theta_t) = sin(theta_i) / eta_rel in the plane of
    incidence on the far side; reflection is the mirror direction; the radiance
    factor is 1/eta_rel^2 on refraction and 1 on reflection; beyond the critical
    angle every choice reflects; the reflection probability equals F."""
    rng = np.random.default_rng(5)
    n_checked_tir = 0
    for _ in range(400):
        ng = _unit(rng.normal(size=3))
        wi = _unit(rng.normal(size=3))
        c = float(np.dot(ng, wi))
        if abs(c) < 1e-3:
            continue
        entering = c > 0
        n = ng if entering else -ng
        eta_rel = eta if entering else 1.0 / eta
        cos_i = abs(c)
        sin_i = math.sqrt(max(0.0, 1.0 - cos_i * cos_i))
        # reflection (u3 = 0 always reflects, F > 0)
        refr, wo, w = oracle_mod.dielectric_sample(ng, wi, eta, 0.0)
        assert not refr and w == 1.0
        assert abs(np.linalg.norm(wo) - 1.0) < 1e-12
        assert abs(np.dot(wo, n) - cos_i) < 1e-12                       # same angle, same side
        assert np.linalg.norm(np.cross(wo + wi, n)) < 1e-12             # wo + wi along n
        # refraction or total internal reflection (u3 just below 1)
        refr, wo, w = oracle_mod.dielectric_sample(ng, wi, eta, 1.0 - 1e-12)
        tir = sin_i / eta_rel >= 1.0
        if tir:
            n_checked_tir += 1
            assert not refr and w == 1.0
            assert abs(np.dot(wo, n) - cos_i) < 1e-12
            continue
        assert refr
        assert abs(np.linalg.norm(wo) - 1.0) < 1e-12
        cos_t = -float(np.dot(wo, n))
        assert cos_t > 0.0                                              # far side
        sin_t = math.sqrt(max(0.0, 1.0 - cos_t * cos_t))
        assert abs(sin_t - sin_i / eta_rel) < 1e-12                     # Snell
        assert abs(np.dot(np.cross(n, wi), wo)) < 1e-12                 # plane of incidence
        # tangential components point the same way (the ray bends, it does not fold back)
        ti = wi - n * cos_i
        to = wo + n * cos_t
        assert np.dot(ti, to) <= 1e-12
        assert abs(w - 1.0 / eta_rel ** 2) < 1e-15
        # the switch between reflection and refraction sits at u3 = F
        F = oracle_mod.fresnel(cos_i, eta_rel)
        assert not oracle_mod.dielectric_sample(ng, wi, eta, F * (1 - 1e-9))[0]
        assert oracle_mod.dielectric_sample(ng, wi, eta, min(F * (1 + 1e-9) + 1e-15, 1 - 1e-15))[0]
    assert n_checked_tir > 20


def _glass_samples(oracle_mod, inside, nee, spp=16, depth=48, eta=1.5, L=1.3):
    sc = S.glass_sphere(eta=eta, env_radiance=L, inside=inside, level=3, width=16, height=16)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], spp=spp, max_depth=depth, seed=31, nee=nee)
    _, sl, _ = oracle_mod.render(osc, r, per_sample=True)
    return sl.reshape(-1, 3), float(np.float32(eta)), float(np.float32(L))


@pytest.mark.parametrize("nee", [False, True])
def test_glass_furnace_outside(oracle_mod, nee):
    """A lossless glass sphere in a uniform sky of radiance L, seen from outside:
    every path that leaves into the sky carries exactly L, whatever the mix of
    reflections and refractions (R + T = 1 and the 1/eta^2 factors cancel on
    the way in and out).  Paths cut off by the depth limit inside the glass are
    the only zeros, and they are rare."""
    x, _, L = _glass_samples(oracle_mod, inside=False, nee=nee)
    esc = x[:, 0] > 0
    assert np.allclose(x[esc], L, rtol=1e-12, atol=0)
    assert np.all(x[~esc] == 0.0)
    assert (~esc).mean() < 0.005


def test_glass_furnace_inside(oracle_mod):
    """Camera inside the glass: the radiance theorem (L / n^2 invariant) gives
    eta^2 L along every path that leaves into the sky.  This fixes the direction
    of the 1/eta^2 radiance scaling, which cancels for an outside observer."""
    x, eta, L = _glass_samples(oracle_mod, inside=True, nee=False)
    esc = x[:, 0] > 0
    assert np.allclose(x[esc], eta * eta * L, rtol=1e-12, atol=0)
    assert esc.mean() > 0.995


# ---------------------------------------------------------------- Russian roulette
@pytest.mark.parametrize("a,R", [(0.5, 1), (0.5, 3), (0.98, 1), (0.7, 2)])
def test_roulette_unbiased_with_stated_continuation(oracle_mod, a, R):
    """White furnace (Le = E and albedo a on every face, BSDF sampling only, depth D)
    with roulette from depth R.  The mean stays E * sum_{k<D} a^k (within 4 sigma).
    A sample's value tells how many vertices m its path reached; the observed
    fraction of paths that continue past vertex k >= R matches
    q_k = min(max(beta_k), 0.95), beta_k being the throughput after sampling at
    vertex k (divided by the earlier q's), and every value lies on the lattice
    of partial sums that this rule produces."""
    E, D = 1.0, 8
    sc = S.furnace(a, E, 32, 32)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], spp=32, max_depth=D, seed=41, rr_depth=R, nee=False)
    _, sl, _ = oracle_mod.render(osc, r, per_sample=True)
    x = sl[..., 0].ravel()
    a32 = float(np.float32(a))
    # unbiased: the roulette-free closed form
    want = E * sum(a32 ** k for k in range(D))
    assert abs(x.mean() - want) < 4 * x.std() / math.sqrt(x.size)
    # lattice of values and continuation probabilities of the stated rule
    beta, value, vals, qs = 1.0, E, [E], []
    for k in range(1, D):
        beta *= a32                      # cosine-sampled diffuse: f cos / pdf = a
        if k >= R:
            q = min(beta, 0.95)
            qs.append((k, q))
            beta /= q
        else:
            qs.append((k, 1.0))
        value += E * beta
        vals.append(value)
    vals = np.array(vals)
    m = np.abs(x[:, None] - vals[None, :]).argmin(axis=1)          # vertices reached - 1
    assert np.allclose(x, vals[m], rtol=1e-12, atol=0)
    assert m.min() == min(R, D) - 1                                  # no roulette before depth R
    for k, q in qs:
        reached = m >= k - 1
        n = int(reached.sum())
        if n < 200:
            break
        cont = (m[reached] >= k).mean()
        assert abs(cont - q) <= 4 * math.sqrt(q * (1 - q) / n) + 1e-12, (k, cont, q)


# ---------------------------------------------------------------- GGX masking
def _phi_integral_of_positive_part(A, B):
    """int_0^{2 pi} max(0, A cos(phi) + B) d phi for A >= 0."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    out = np.where(B >= A, 2 * np.pi * B, 0.0)
    mid = (B < A) & (B > -A)
    with np.errstate(invalid="ignore", divide="ignore"):
        p0 = np.arccos(np.clip(-B / np.where(A > 0, A, 1.0), -1.0, 1.0))
    return np.where(mid, 2.0 * (A * np.sin(p0) + B * p0), out)


@pytest.mark.parametrize("alpha", [0.1, 0.3, 0.5, 1.0])
def test_ggx_weak_white_furnace(oracle_mod, alpha):
    """Heitz (2014): with a correct Smith masking function,
    int_{S^2} D(h) G1(o) / (4 |o.n|) d omega_i = 1 for every outgoing o, where h is
    the half vector of o and i.  With d omega_i = 4 (o.h) d omega_h this is
    G1(o) int_{o.h > 0} D(h) (o.h) d omega_h / cos(theta_o) = 1.  The integral is
    taken by quadrature over the half-vector hemisphere, with the azimuth done in
    closed form; the same quadrature also checks int D cos(theta_h) = 1."""
    N = 20000
    u = (np.arange(N) + 0.5) / N
    # x = 1 - (1 - u)^2 removes the (1 - x)^(-1/2) end point behaviour; then
    # tan^2(theta_h) = alpha^2 x / (1 - x) places nodes where D has its mass.
    x = 1.0 - (1.0 - u) ** 2
    dxdu = 2.0 * (1.0 - u)
    t = alpha * alpha * x / (1.0 - x)
    cos_h = 1.0 / np.sqrt(1.0 + t)
    sin_h = np.sqrt(np.maximum(0.0, 1.0 - cos_h * cos_h))
    dcos_dx = 0.5 * (1.0 + t) ** -1.5 * alpha * alpha / (1.0 - x) ** 2
    w = dcos_dx * dxdu / N                                            # |d cos(theta_h)| per node
    D = np.array([oracle_mod.ggx_terms(alpha, c, 1.0)[0] for c in cos_h])
    norm = np.sum(D * cos_h * w) * 2 * np.pi
    assert abs(norm - 1.0) < 2e-4, norm
    for th_deg in (0.0, 30.0, 60.0, 80.0, 88.0):
        th = math.radians(th_deg)
        co, so = math.cos(th), math.sin(th)
        G1 = oracle_mod.ggx_terms(alpha, 1.0, co)[1]
        # o.h = so sin_h cos(phi) + co cos_h, integrated over phi in closed form
        proj = np.sum(D * _phi_integral_of_positive_part(so * sin_h, co * cos_h) * w)
        val = G1 * proj / co
        assert abs(val - 1.0) < 2e-4, (alpha, th_deg, val)


# ---------------------------------------------------------------- training records
@pytest.mark.parametrize("a,D", [(0.5, 5), (0.8, 4)])
def test_training_targets_in_the_white_furnace(oracle_mod, a, D):
    """In the white furnace without light sampling, the radiance that leaves a
    vertex reached by segment k toward the previous vertex, minus its own
    emission, is E * sum_{m=1}^{D-k} a^m with zero variance.  Each record's
    target, (L_path - L_before) / beta, must equal that exactly."""
    E = 1.0
    sc = S.furnace(a, E, 8, 8)
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], spp=4, max_depth=D, seed=47, nee=False)
    raw, tgt, meta = oracle_mod.train_records(osc, r, cap=8 * 8 * 4 * D)
    assert raw.shape[0] == 8 * 8 * 4 * (D - 1)                      # one record per vertex k < D
    a32 = float(np.float32(a))
    depth = meta[:, 1]
    want = np.array([E * sum(a32 ** m for m in range(1, D - k + 1)) for k in depth])
    assert np.allclose(tgt, want[:, None], rtol=1e-12, atol=0)
    # every depth 1 .. D-1 is present for every sample
    assert set(depth.tolist()) == set(range(1, D))
