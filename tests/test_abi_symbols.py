"""The C-ABI library builds, loads without a GPU and exports every symbol include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:int|void|const char\*)\s+(pt_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2202_01284_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("pt_scene_create", "pt_bvh_build", "pt_render_forward", "pt_render_backward",
                     "pt_scene_destroy", "pt_status_string", "pt_last_device_status"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    from paper_2202_01284_gb300 import abi
    L = abi.load(libpath)
    assert L.pt_status_string(0) == b"ok"
    assert b"argument" in L.pt_status_string(abi.PT_ERR_ARG)


def test_null_arguments_rejected_without_gpu(libpath):
    from paper_2202_01284_gb300 import abi
    L = abi.load(libpath)
    h = ctypes.c_void_p()
    assert L.pt_scene_create(None, ctypes.byref(h)) == abi.PT_ERR_ARG
    assert L.pt_bvh_build(None, None) == abi.PT_ERR_ARG
    assert L.pt_render_forward(None, None, None, None, None) == abi.PT_ERR_ARG
    assert L.pt_render_backward(None, None, None, None, None, None) == abi.PT_ERR_ARG
