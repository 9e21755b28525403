"""User meshes: the OBJ reader and mesh_scene (host side only)."""
import numpy as np

from paper_2202_01284_gb300 import scenes as S

OBJ = """
# a unit quad (one polygon) and a triangle in a second group, with uvs
v 0 0 0
v 1 0 0
v 1 1 0
v 0 1 0
vt 0 0
vt 1 0
vt 1 1
vt 0 1
o quad
f 1/1 2/2 3/3 4/4
g tri
v 0 0 1
f -1 1 2
"""


def test_obj_fan_groups_and_uvs():
    v, uv, grp, names = S.load_obj(OBJ)
    assert v.shape == (3, 3, 3) and uv.shape == (3, 3, 2)
    assert names == ["quad", "tri"] and list(grp) == [0, 0, 1]
    np.testing.assert_array_equal(v[0], [[0, 0, 0], [1, 0, 0], [1, 1, 0]])
    np.testing.assert_array_equal(v[1], [[0, 0, 0], [1, 1, 0], [0, 1, 0]])
    np.testing.assert_array_equal(v[2], [[0, 0, 1], [0, 0, 0], [1, 0, 0]])
    np.testing.assert_array_equal(uv[1], [[0, 0], [1, 1], [0, 1]])
    assert not uv[2].any()


def test_mesh_scene_renders_on_the_oracle(oracle_mod):
    v, uv, grp, _ = S.load_obj(OBJ)
    cam = S.Camera((0.5, 0.5, 3.0), (0.5, 0.5, 0.0), (0, 1, 0), 40.0, 8, 8)
    env = np.ones((8, 16, 4), np.float32)
    sc = S.mesh_scene(v, uv, grp, albedo=[[0.5, 0.5, 0.5], [0.2, 0.3, 0.4]], env=env, cameras=[cam])
    assert sc.n_shapes == 2 and sc.n_tris == 3
    img = oracle_mod.render(oracle_mod.OracleScene(sc), oracle_mod.render_in(cam, 4, 3, 1))
    assert img.shape == (8, 8, 3) and np.isfinite(img).all() and img.max() > 0


def test_pfm_round_trip(tmp_path):
    from paper_2202_01284_gb300.render import load_pfm, save_pfm
    img = np.random.default_rng(0).random((5, 7, 3)).astype(np.float32)
    p = str(tmp_path / "img.pfm")
    save_pfm(p, img)
    back = load_pfm(p)
    assert back.shape == (5, 7, 3) and np.array_equal(back, img)
    with open(p, "rb") as f:
        assert f.readline() == b"PF\n" and f.readline() == b"7 5\n"
