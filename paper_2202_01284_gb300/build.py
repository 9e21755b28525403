"""Build of the in-tree CUDA library ``libptgb.so`` (nvcc, sm_103a only).

Each translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and linked with
``-shared``; the result lives next to this file and is loaded through ctypes.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libptgb.so")
OBJDIR = os.path.join(HERE, "_build")

CU_SOURCES = ["pt_render.cu", "pt_scene.cu", "pt_nrc.cu", "pt_nrc_tc.cu", "pt_wavefront.cu", "pt_ckpt.cu",
              "pt_reparam.cu", "pt_probe.cu"]
CPP_SOURCES = ["bvh_build.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Per-source floating-point flags.  In the megakernel sources device divisions a / b
# and square roots are the approximate ones (at most 2 ulp / the hardware square root):
# measured 3.4 % and 1.7 % of the path tracer's step.  The triangle test's 1 / det
# uses __frcp_rn everywhere (hit decisions as under IEEE division); the ray's inverse
# direction, which only the padded box tests use, the hardware reciprocal.  The reparameterized source keeps IEEE division: with the approximate
# one its glossy log-derivatives and vertex-mode tangents moved by up to 1.6e-3
# relative against the FP64 reference (the warp estimator's own ratios of sums,
# written as __fdiv_rn / __frcp_rn, were not the cause).  The cache MLP keeps IEEE
# division and square root.
_MEGA_FLAGS = ["-prec-div=false", "-prec-sqrt=false"]
SOURCE_FLAGS = {"pt_render.cu": _MEGA_FLAGS, "pt_wavefront.cu": _MEGA_FLAGS, "pt_ckpt.cu": _MEGA_FLAGS}


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES]


def _deps():
    out = _sources()
    for f in os.listdir(CSRC):
        if f.endswith((".h", ".cuh")):
            out.append(os.path.join(CSRC, f))
    out.append(os.path.join(INCLUDE, "pt.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False, defines=()) -> str:
    """defines: extra preprocessor definitions ("NAME=value"), e.g. the register caps
    PT_FWD_REGS / PT_ADJ_MIN_BLOCKS / PT_REPLAY_MIN_BLOCKS for tuning."""
    if not force and not defines and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJDIR, exist_ok=True)
    common = ["-O3", "-std=c++20", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + [f"-D{d}" for d in defines]

    def compile_one(src):
        obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
        if src.endswith(".cu"):
            flags = SOURCE_FLAGS.get(os.path.basename(src), [])
            cmd = [nvcc, *ARCH, "-lineinfo", "--expt-relaxed-constexpr", *flags, *common, "-c", src, "-o", obj]
            if ptxas_verbose:
                cmd += ["-Xptxas", "-v"]
        else:
            cmd = [nvcc, *common, "-x", "c++", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(_sources())) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose or ptxas_verbose:
        for _, err in results:
            if err:
                print(err)
    objs = [o for o, _ in results]
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, ptxas_verbose="-v" in sys.argv))
