"""Host-side checks of the library's BVH builder (no GPU): index bounds, triangle
permutation, box containment and a replay of the 8-wide traversal rules vs brute force."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2202_01284_gb300 import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_01284_gb300", "csrc")


@pytest.fixture(scope="module", params=["dp", "greedy"])
def harness(request):
    """The builder as shipped (8-wide tree by the cost-optimal collapse) and with the
    greedy largest-area collapse it falls back to for trees deeper than the traversal
    stack."""
    flags = [] if request.param == "dp" else ["-DPT_WIDE_COLLAPSE_DP=0"]
    out = os.path.join(tempfile.mkdtemp(prefix="bvhh"), "libbvhh.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, *flags, "-o", out,
                    os.path.join(HERE, "bvh_harness.cpp"), os.path.join(CSRC, "bvh_build.cpp")], check=True)
    lib = ctypes.CDLL(out)
    lib.check_bvh.restype = ctypes.c_int
    lib.check_bvh.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                              ctypes.c_void_p]
    return lib


def _rays(n, seed, center, spread):
    rng = np.random.default_rng(seed)
    o = center + rng.uniform(-spread, spread, size=(n, 3))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.ascontiguousarray(np.concatenate([o, d], 1).astype(np.float32))


@pytest.mark.parametrize("case", ["cornell", "soup", "spheres", "tiny"])
def test_bvh_layouts(harness, case):
    if case == "cornell":
        V = S.cornell().vertices
        rays = _rays(3000, 1, np.array([0, 1, 0]), 0.9)
    elif case == "soup":
        rng = np.random.default_rng(2)
        c = rng.uniform(-1, 1, size=(2000, 1, 3))
        V = (c + 0.05 * rng.normal(size=(2000, 3, 3))).astype(np.float32)
        rays = _rays(3000, 3, np.zeros(3), 1.2)
    elif case == "spheres":
        V = S.spheres(n_spheres=6, level=3, grid=(3, 2), ground_quads=16, tex_res=16).vertices
        rays = _rays(2000, 4, np.array([0, 1.0, 0]), 3.0)
    else:
        V = S.cornell().vertices[:2]
        rays = _rays(500, 5, np.array([0, 0.5, 0.5]), 1.0)
    V = np.ascontiguousarray(V, np.float32)
    stats = np.zeros(4, np.int64)
    bad = harness.check_bvh(V.ctypes.data, V.shape[0], rays.ctypes.data, rays.shape[0], 3, stats.ctypes.data)
    assert bad == 0
    assert stats[1] == 0, f"{stats[1]} traversal mismatches vs brute force"
    assert stats[0] >= 1
