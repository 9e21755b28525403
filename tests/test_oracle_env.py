"""Pins of the oracle's environment-radiance derivatives (CPU only).

With sampling detached (the scene's map drives the env importance sampler; only
the radiance used for shading moves), every sample is a sum of terms each linear
in one env pixel, so the fixed-seed image is linear in the env radiance and a
central difference is exact up to rounding.  The stored-tape gradient, the dual
numbers and the forward-mode tangent are pinned against it and each other.
"""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S


@pytest.fixture(scope="module")
def env_scene():
    sc = S.spheres(n_spheres=4, level=1, grid=(2, 2), ground_quads=4, tex_res=64, width=24, height=18,
                   env_size=(32, 16))
    return sc


def _rin(oracle_mod, sc, env=None, spp=4, seed=3):
    return oracle_mod.render_in(sc.cameras[0], spp, 5, seed, 2, True, env_radiance=env)


def test_override_equal_to_scene_map_changes_nothing(oracle_mod, env_scene):
    sc = env_scene
    osc = oracle_mod.OracleScene(sc)
    a = oracle_mod.render(osc, _rin(oracle_mod, sc))
    b = oracle_mod.render(osc, _rin(oracle_mod, sc, env=sc.env.astype(np.float64)))
    assert np.array_equal(a, b)


def test_env_jvp_matches_central_difference(oracle_mod, env_scene):
    sc = env_scene
    osc = oracle_mod.OracleScene(sc)
    base = sc.env.astype(np.float64)
    rng = np.random.default_rng(7)
    v = rng.normal(size=base.shape)
    v[..., 3] = 0
    h = 0.25
    Ip = oracle_mod.render(osc, _rin(oracle_mod, sc, env=base + h * v))
    Im = oracle_mod.render(osc, _rin(oracle_mod, sc, env=base - h * v))
    fd = (Ip - Im) / (2 * h)
    img, dot = oracle_mod.render_jvp(osc, _rin(oracle_mod, sc), t_env=v)
    scale = np.abs(dot).max()
    assert scale > 0
    assert np.abs(fd - dot).max() < 1e-10 * scale
    # linear: one-sided difference with a large step is exact too
    I2 = oracle_mod.render(osc, _rin(oracle_mod, sc, env=base + 3.0 * v))
    assert np.abs((I2 - img) / 3.0 - dot).max() < 1e-10 * scale


def test_env_gradient_tape_dual_and_identity(oracle_mod, env_scene):
    sc = env_scene
    osc = oracle_mod.OracleScene(sc)
    r = _rin(oracle_mod, sc)
    rng = np.random.default_rng(8)
    img = oracle_mod.render(osc, r)
    gi = rng.normal(size=img.shape)
    ga, gt, gr, ge = oracle_mod.grad_tape(osc, r, gi, env=True)
    assert ge.shape == sc.env.shape and np.abs(ge).max() > 0
    assert not ge[..., 3].any()
    # dual numbers on the env pixels with the largest gradients
    flat = np.abs(ge[..., :3]).reshape(-1)
    top = np.argsort(flat)[-8:]
    sel = [(3, int(i // 3), int(i % 3), 0) for i in top]
    gd = oracle_mod.grad_dual(osc, r, gi, sel)
    want = np.array([ge.reshape(-1, 4)[p, c] for (_, p, c, _) in sel])
    assert np.allclose(gd, want, rtol=1e-10, atol=1e-14 * np.abs(want).max())
    # <gi, J v> = <J^T gi, v> for a random env direction (and mixed with texels)
    v = rng.normal(size=sc.env.shape)
    v[..., 3] = 0
    vt = rng.normal(size=sc.textures[0].shape)
    vt[..., 3] = 0
    _, dot = oracle_mod.render_jvp(osc, r, t_textures=[vt], t_env=v)
    lhs = float((gi * dot).sum())
    rhs = float((ge * v).sum() + (gt[0] * vt).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), abs(rhs))


def test_env_gradient_without_nee(oracle_mod, env_scene):
    """With light sampling off, env radiance enters only where paths escape: the
    gradient is the BSDF-sampled escape weight, still linear (central difference)."""
    sc = env_scene
    osc = oracle_mod.OracleScene(sc)
    r = oracle_mod.render_in(sc.cameras[0], 4, 4, 5, -1, False)
    img = oracle_mod.render(osc, r)
    gi = np.ones_like(img)
    _, _, _, ge = oracle_mod.grad_tape(osc, r, gi, env=True)
    base = sc.env.astype(np.float64)
    rng = np.random.default_rng(9)
    v = rng.normal(size=base.shape)
    v[..., 3] = 0
    Ip = oracle_mod.render(osc, oracle_mod.render_in(sc.cameras[0], 4, 4, 5, -1, False, env_radiance=base + v))
    assert abs(float((Ip - img).sum()) - float((ge * v).sum())) <= 1e-10 * abs(float((ge * v).sum()))
