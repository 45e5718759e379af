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


def test_track_step_upload_validates_before_any_cuda_call(libpath):
    """gs_track_step_upload refuses a missing src, a zero iteration count, and (reading the
    frame in place, targets NULL) a src without rgb or depth, before any CUDA call."""
    from paper_2408_05635_gb300 import gs
    lib = ctypes.CDLL(libpath)
    lib.gs_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    lib.gs_track_step_upload.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(gs.gs_host_targets), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.gs_create(ctypes.byref(h), None) == 0
    frame = (ctypes.c_float * 8)()
    result = (ctypes.c_double * 8)()
    addr = ctypes.addressof(frame)
    ok_src = gs.gs_host_targets(addr, addr, None, ctypes.addressof(result))
    no_rgb = gs.gs_host_targets(None, addr, None, None)
    no_depth = gs.gs_host_targets(addr, None, None, None)
    call = lambda src, iters: lib.gs_track_step_upload(h, None, None, None, src, None, None, None, iters, None, 0,
                                                       None)
    assert call(None, 1) == 1
    assert call(ctypes.byref(ok_src), 0) == 1
    assert call(ctypes.byref(no_rgb), 1) == 1
    assert call(ctypes.byref(no_depth), 1) == 1
    lib.gs_destroy.argtypes = [ctypes.c_void_p]
    lib.gs_destroy(h)


def _ctx(lib, cfg=None):
    lib.gs_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]
    h = ctypes.c_void_p()
    st = lib.gs_create(ctypes.byref(h), cfg)
    return st, h


def test_schedule_host_logic(libpath):
    """gs_get_schedule / gs_set_schedule (host-only calls): the default schedule, the sets
    of valid values, and a workspace size that does not depend on the schedule."""
    from paper_2408_05635_gb300 import gs
    lib = ctypes.CDLL(libpath)
    lib.gs_get_schedule.argtypes = [ctypes.c_void_p, ctypes.POINTER(gs.gs_schedule)]
    lib.gs_set_schedule.argtypes = [ctypes.c_void_p, ctypes.POINTER(gs.gs_schedule)]
    lib.gs_workspace_size.argtypes = [ctypes.c_void_p, ctypes.POINTER(gs.gs_problem), ctypes.POINTER(ctypes.c_size_t)]
    lib.gs_destroy.argtypes = [ctypes.c_void_p]
    st, h = _ctx(lib)
    assert st == 0
    s = gs.gs_schedule()
    assert lib.gs_get_schedule(h, ctypes.byref(s)) == 0
    assert gs.schedule_dict(s) == {"tile_w": 16, "tile_h": 16, "sub_buckets": 4, "fwd_batch": 256, "bwd_batch": 256,
                                   "flags": 0}
    cams = (gs.gs_camera * 3)(gs.gs_camera(525, 525, 319.5, 239.5, 640, 480), gs.gs_camera(100, 100, 10, 10, 37, 23),
                              gs.gs_camera(600, 600, 599.5, 339.5, 1200, 680))
    prob = gs.gs_problem(50000, 3, 0, ctypes.cast(cams, ctypes.POINTER(gs.gs_camera)), 1 << 20, 0)
    sizes = set()
    good = [(16, 16, 4, 256, 256), (32, 8, 2, 256, 64), (16, 8, 1, 128, 128), (8, 8, 4, 64, 64), (8, 32, 2, 256, 128),
            (32, 4, 4, 128, 64), (16, 4, 1, 64, 64), (8, 16, 2, 128, 64)]
    for v in good:
        assert lib.gs_set_schedule(h, ctypes.byref(gs.gs_schedule(*v, 0))) == 0, v
        assert lib.gs_get_schedule(h, ctypes.byref(s)) == 0 and tuple(gs.schedule_dict(s).values()) == v + (0,)
        n = ctypes.c_size_t(0)
        assert lib.gs_workspace_size(h, ctypes.byref(prob), ctypes.byref(n)) == 0
        sizes.add(n.value)
    assert len(sizes) == 1  # the layout has room for every tile shape
    bad = [(16, 16, 3, 256, 256), (16, 16, 4, 100, 256), (16, 16, 4, 256, 512), (8, 8, 4, 128, 64),
           (16, 8, 4, 128, 256), (4, 16, 4, 64, 64), (64, 4, 4, 64, 64), (8, 4, 4, 64, 64), (32, 16, 4, 256, 256),
           (12, 16, 4, 64, 64), (16, 16, 0, 64, 64)]
    last = gs.gs_schedule(*good[-1], 0)
    for v in bad:
        assert lib.gs_set_schedule(h, ctypes.byref(gs.gs_schedule(*v, 0))) == 1, v
    assert lib.gs_set_schedule(h, ctypes.byref(gs.gs_schedule(16, 16, 4, 256, 256, 6))) == 1  # unknown flags
    # the fused tracking kernel needs one batch depth for both walks
    assert lib.gs_set_schedule(h, ctypes.byref(gs.gs_schedule(16, 16, 4, 256, 128, gs.GS_SCHED_FUSED))) == 1
    assert lib.gs_get_schedule(h, ctypes.byref(s)) == 0 and gs.schedule_dict(s) == gs.schedule_dict(last)
    assert lib.gs_set_schedule(h, ctypes.byref(gs.gs_schedule(16, 8, 2, 128, 128, gs.GS_SCHED_FUSED))) == 0
    assert lib.gs_get_schedule(h, ctypes.byref(s)) == 0 and s.flags == gs.GS_SCHED_FUSED
    assert lib.gs_destroy(h) == 0


def test_config_tile_sets_the_initial_schedule(libpath):
    from paper_2408_05635_gb300 import gs
    lib = ctypes.CDLL(libpath)
    lib.gs_get_schedule.argtypes = [ctypes.c_void_p, ctypes.POINTER(gs.gs_schedule)]
    lib.gs_destroy.argtypes = [ctypes.c_void_p]
    lib.gs_default_config.argtypes = [ctypes.POINTER(gs.gs_config)]
    for (w, hgt), ok in [((16, 8), True), ((8, 8), True), ((32, 8), True), ((16, 16), True), ((4, 4), False),
                         ((64, 4), False), ((24, 8), False)]:
        cfg = gs.gs_config()
        lib.gs_default_config(ctypes.byref(cfg))
        cfg.tile_w, cfg.tile_h = w, hgt
        st, h = _ctx(lib, ctypes.byref(cfg))
        if not ok:
            assert st == 7 and not h.value  # GS_ERR_UNSUPPORTED
            continue
        assert st == 0
        s = gs.gs_schedule()
        assert lib.gs_get_schedule(h, ctypes.byref(s)) == 0
        nb = min(256, w * hgt)
        assert gs.schedule_dict(s) == {"tile_w": w, "tile_h": hgt, "sub_buckets": 4, "fwd_batch": nb, "bwd_batch": nb,
                                       "flags": 0}
        lib.gs_destroy(h)
