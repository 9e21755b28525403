"""Pins of the oracle's forward-mode image derivative (CPU only).

image_dot = d/d eps image(params + eps v) with sampling detached.  It is pinned
by (1) finite differences where sampling does not depend on the parameter
(albedo rows and texels enter the estimator polynomially), (2) the identity
<grad_image, J v> = <J^T grad_image, v> against the stored-tape reverse mode,
an independent derivative engine (this covers roughness, whose sampling the
detached derivative ignores), and (3) linearity in v.
"""
import numpy as np

from paper_2202_01284_gb300 import scenes as S


def _richardson_image(oracle_mod, make_scene, r, base, v, h=2.0 ** -9):
    """Richardson-extrapolated central difference of the fixed-seed image along v.
    Returns (estimate, exact direction): the float32 scene stores the perturbed
    values, so the direction actually applied is recomputed from them."""
    ests, dirs = [], []
    for hh in (h, h / 2):
        p = (base + hh * v).astype(np.float32)
        m = (base - hh * v).astype(np.float32)
        Ip = oracle_mod.render(oracle_mod.OracleScene(make_scene(p)), r)
        Im = oracle_mod.render(oracle_mod.OracleScene(make_scene(m)), r)
        ests.append((Ip - Im) / (2 * hh))
        dirs.append((p.astype(np.float64) - m.astype(np.float64)) / (2 * hh))
    return (4 * ests[1] - ests[0]) / 3, dirs


def test_jvp_albedo_direction_matches_finite_differences(oracle_mod):
    sc = S.cornell(width=24, height=24)
    r = oracle_mod.render_in(sc.cameras[0], 2, 4, seed=11)
    rng = np.random.default_rng(3)
    # dyadic direction: base +- h v is exact in float32 for these h
    v = rng.integers(-4, 5, size=sc.albedo.shape).astype(np.float64) / 4
    base = sc.albedo.astype(np.float64)
    fd, dirs = _richardson_image(oracle_mod, lambda a: sc.with_params(albedo=a), r, base, v)
    assert all(np.array_equal(d, v) for d in dirs)
    img, dot = oracle_mod.render_jvp(oracle_mod.OracleScene(sc), r, t_albedo=v)
    assert np.array_equal(img, oracle_mod.render(oracle_mod.OracleScene(sc), r))
    scale = np.abs(dot).max()
    assert scale > 0
    assert np.abs(fd - dot).max() < 1e-8 * scale


def test_jvp_texel_direction_matches_finite_differences(oracle_mod):
    sc = S.cornell96(width=20, height=20, tex_res=64)
    # texel values on a 2^-12 grid so that tex +- h v is exact in float32
    tex = np.round(sc.textures[0].astype(np.float64) * 4096) / 4096
    sc = sc.with_params(textures=[tex])
    r = oracle_mod.render_in(sc.cameras[0], 2, 4, seed=5)
    rng = np.random.default_rng(4)
    v = np.zeros_like(tex)
    v[..., :3] = rng.integers(-2, 3, size=tex[..., :3].shape) / 2
    fd, dirs = _richardson_image(oracle_mod, lambda t: sc.with_params(textures=[t]), r, tex, v)
    assert all(np.array_equal(d, v) for d in dirs)
    _, dot = oracle_mod.render_jvp(oracle_mod.OracleScene(sc), r, t_textures=[v])
    scale = np.abs(dot).max()
    assert scale > 0
    assert np.abs(fd - dot).max() < 1e-8 * scale


def test_jvp_vjp_dot_product_identity(oracle_mod):
    """<gi, J v> == <J^T gi, v> with J^T gi from the stored-tape adjoint, for a
    mixed direction over albedo rows, texels and roughness entries."""
    sc = S.cornell96(width=20, height=20, tex_res=64)
    r = oracle_mod.render_in(sc.cameras[0], 3, 5, seed=8)
    osc = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(5)
    va = rng.normal(size=sc.albedo.shape) if sc.albedo.size else None
    vt = rng.normal(size=sc.textures[0].shape)
    vt[..., 3] = 0
    vr = rng.normal(size=sc.roughness.shape)
    assert sc.roughness.size > 0
    img, dot = oracle_mod.render_jvp(osc, r, t_albedo=va, t_textures=[vt], t_rough=vr)
    gi = rng.normal(size=img.shape)
    ga, gt, gr = oracle_mod.grad_tape(osc, r, gi)
    lhs = float((gi * dot).sum())
    rhs = float((gt[0][..., :3] * vt[..., :3]).sum() + (gr * vr).sum())
    if va is not None:
        rhs += float((ga * va).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs), 1e-30)
    # roughness alone is a real (non-zero) part of the check
    _, dot_r = oracle_mod.render_jvp(osc, r, t_rough=vr)
    assert abs(float((gi * dot_r).sum()) - float((gr * vr).sum())) <= 1e-10 * abs(float((gr * vr).sum()))
    assert abs(float((gr * vr).sum())) > 0


def test_jvp_is_linear_in_direction(oracle_mod):
    sc = S.cornell(width=16, height=16)
    r = oracle_mod.render_in(sc.cameras[0], 2, 4, seed=2)
    osc = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(6)
    v1, v2 = rng.normal(size=sc.albedo.shape), rng.normal(size=sc.albedo.shape)
    _, d1 = oracle_mod.render_jvp(osc, r, t_albedo=v1)
    _, d2 = oracle_mod.render_jvp(osc, r, t_albedo=v2)
    _, d12 = oracle_mod.render_jvp(osc, r, t_albedo=2 * v1 - 3 * v2)
    assert np.allclose(d12, 2 * d1 - 3 * d2, rtol=1e-12, atol=1e-14 * np.abs(d12).max())
    _, d0 = oracle_mod.render_jvp(osc, r)
    assert not d0.any()
