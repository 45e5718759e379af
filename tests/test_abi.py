"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry
point include/gs.h declares (no compute calls: those need a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gs_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2408_05635_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    names = declared_entry_points()
    for required in ("gs_project", "gs_forward", "gs_backward", "gs_track_step", "gs_workspace_size",
                     "gs_create", "gs_destroy", "gs_sync_status"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gs_[a-z_]+)\b", out))
    missing = [n for n in declared_entry_points() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_host_only_calls(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gs_status_string.restype = ctypes.c_char_p
    assert lib.gs_status_string(5) == b"GS_ERR_CAPACITY"
    # argument validation happens before any CUDA call
    lib.gs_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.gs_create(ctypes.byref(h), None) == 0
    lib.gs_workspace_size.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gs_workspace_size(h, None, None) == 1
    lib.gs_destroy.argtypes = [ctypes.c_void_p]
    assert lib.gs_destroy(h) == 0


def test_workspace_size_validation(libpath):
    import numpy as np  # noqa: F401
    from paper_2408_05635_gb300 import gs
    lib = ctypes.CDLL(libpath)
    lib.gs_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    lib.gs_workspace_size.argtypes = [ctypes.c_void_p, ctypes.POINTER(gs.gs_problem), ctypes.POINTER(ctypes.c_size_t)]
    h = ctypes.c_void_p()
    assert lib.gs_create(ctypes.byref(h), None) == 0
    cams = (gs.gs_camera * 2)(gs.gs_camera(525, 525, 319.5, 239.5, 640, 480), gs.gs_camera(100, 100, 10, 10, 20, 20))
    prob = gs.gs_problem(200000, 2, 0, ctypes.cast(cams, ctypes.POINTER(gs.gs_camera)), 1 << 22, 0)
    n = ctypes.c_size_t(0)
    assert lib.gs_workspace_size(h, ctypes.byref(prob), ctypes.byref(n)) == 0
    # record slots 2N x 96 B, pairs 12 B each, pixels 28 B each: a lower bound on the layout
    assert n.value >= 2 * 200000 * 96 + (1 << 22) * 12 + (640 * 480 + 400) * 28
    bad = gs.gs_problem(1000, 2, 0, ctypes.cast(cams, ctypes.POINTER(gs.gs_camera)), 1 << 22, 5)
    assert lib.gs_workspace_size(h, ctypes.byref(bad), ctypes.byref(n)) == 1  # reserved field
    bad = gs.gs_problem(1 << 31, 4, 0, ctypes.cast(cams, ctypes.POINTER(gs.gs_camera)), 1 << 22, 0)
    assert lib.gs_workspace_size(h, ctypes.byref(bad), ctypes.byref(n)) == 1
    bad = gs.gs_problem(1000, 2, 0, ctypes.cast(cams, ctypes.POINTER(gs.gs_camera)), 0, 0)
    assert lib.gs_workspace_size(h, ctypes.byref(bad), ctypes.byref(n)) == 1
    lib.gs_destroy.argtypes = [ctypes.c_void_p]
    lib.gs_destroy(h)
