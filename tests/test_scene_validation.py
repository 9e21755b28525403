"""Host-side fault injection: malformed scenes are rejected with PT_ERR_ARG before
any device call (so these run on machines without a GPU)."""
import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S


@pytest.fixture(scope="module")
def abi():
    from paper_2202_01284_gb300 import abi, build
    build.build()
    abi.load()
    return abi


def _expect_arg_error(abi, sc):
    with pytest.raises(abi.PtError) as e:
        abi.pt_scene_create(sc)
    assert e.value.code == abi.PT_ERR_ARG


def test_nonfinite_geometry_rejected(abi):
    for bad in (np.nan, np.inf, -np.inf):
        sc = S.cornell(width=8, height=8)
        sc.vertices = sc.vertices.copy()
        sc.vertices[3, 1, 2] = bad
        _expect_arg_error(abi, sc)
        sc = S.cornell(width=8, height=8)
        sc.uvs = sc.uvs.copy()
        sc.uvs[5, 2, 0] = bad
        _expect_arg_error(abi, sc)


def test_bad_emission_and_environment_rejected(abi):
    sc = S.cornell(width=8, height=8)
    sc.emission = sc.emission.copy()
    sc.emission[0, 1] = -1.0
    _expect_arg_error(abi, sc)
    sc = S.cornell(width=8, height=8)
    sc.emission = sc.emission.copy()
    sc.emission[0, 0] = np.nan
    _expect_arg_error(abi, sc)
    sc = S.spheres(n_spheres=2, level=0, grid=(2, 1), ground_quads=2, tex_res=16, width=8, height=8, env_size=(8, 4))
    sc.env = sc.env.copy()
    sc.env[1, 2, 0] = np.inf
    _expect_arg_error(abi, sc)


def test_zero_area_emitter_rejected(abi):
    sc = S.cornell(width=8, height=8)
    sc.vertices = sc.vertices.copy()
    emitting = np.where(sc.emission[sc.tri_shape].max(axis=1) > 0)[0]
    assert emitting.size > 0
    for t in emitting:  # collapse every emitting triangle to a point
        sc.vertices[t, 1] = sc.vertices[t, 0]
        sc.vertices[t, 2] = sc.vertices[t, 0]
    _expect_arg_error(abi, sc)


def test_bad_material_scalars_rejected(abi):
    sc = S.cornell(width=8, height=8)
    sc.alpha = sc.alpha.copy()
    sc.alpha[0] = np.nan
    _expect_arg_error(abi, sc)
