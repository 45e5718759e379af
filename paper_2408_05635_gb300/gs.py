"""ctypes binding of the C ABI in include/gs.h (argument marshalling only).

Every entry point keeps its C name (``gs_project``, ``gs_forward``, ``gs_backward``,
``gs_track_step`` ...) and takes torch CUDA tensors where the C function takes device
pointers.  All compute runs in the CUDA library ``_build/libgsgb.so``; there is no CPU
or PyTorch fallback: loading fails with an error if the library is missing or no CUDA
device is present.

``Rasterizer`` adds the bookkeeping a Python caller needs: it owns the context, sizes
and allocates the workspace (a torch uint8 tensor) and can measure the pair and record
counts of a scene with one sizing pass.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
from typing import Sequence

import numpy as np
import torch

from . import build as _build

c_void_p, c_int32, c_int64, c_uint32, c_double, c_float, c_size_t = (
    ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double, ctypes.c_float,
    ctypes.c_size_t)

GS_F32, GS_BF16, GS_F16 = 0, 1, 2
_STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_OOM", 4: "GS_ERR_WORKSPACE",
           5: "GS_ERR_CAPACITY", 6: "GS_ERR_TIMEOUT", 7: "GS_ERR_UNSUPPORTED", 8: "GS_ERR_STATE"}
GS_ERR_CAPACITY = 5
ERR_RECORDS, ERR_PAIRS, ERR_TIMEOUT = 1, 2, 4


class gs_gaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("quats", c_void_p), ("log_scales", c_void_p),
                ("opacity_logits", c_void_p), ("rgb", c_void_p), ("dtype_attr", c_int32),
                ("reserved", c_int32), ("n", c_int64)]


class gs_gaussians_grad(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("quats", c_void_p), ("log_scales", c_void_p),
                ("opacity_logits", c_void_p), ("rgb", c_void_p)]


class gs_camera(ctypes.Structure):
    _fields_ = [("fx", c_double), ("fy", c_double), ("cx", c_double), ("cy", c_double),
                ("width", c_int32), ("height", c_int32)]


class gs_targets(ctypes.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("depth_prior", c_void_p)]


class gs_host_targets(ctypes.Structure):
    _fields_ = [("rgb", c_void_p), ("depth", c_void_p), ("depth_prior", c_void_p), ("result", c_void_p)]


class gs_config(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32)] + [
        (n, c_float) for n in ("alpha_min", "alpha_max", "t_min", "dilation", "z_near", "jac_clip", "sil_thresh",
                               "w_rgb", "w_depth", "w_vis", "w_prior")] + [
        (n, c_double) for n in ("lr_rot", "lr_trans", "beta1", "beta2", "eps")]


class gs_map(ctypes.Structure):
    _fields_ = [(n, c_void_p) for n in ("means", "quats", "log_scales", "opacity_logits", "rgb", "lowp_quats",
                                         "lowp_log_scales", "lowp_opacity_logits", "lowp_rgb")] + [
        ("lowp_dtype", c_int32), ("reserved", c_int32), ("capacity", c_int64), ("adam_state", c_void_p)]


class gs_map_config(ctypes.Structure):
    _fields_ = [(n, c_double) for n in ("lr_means", "lr_quats", "lr_log_scales", "lr_opacity_logits", "lr_rgb",
                                        "beta1", "beta2", "eps")] + [("sil_add", c_float), ("opacity_min", c_float)]


class gs_problem(ctypes.Structure):
    _fields_ = [("n_gaussians", c_int64), ("n_views", c_int32), ("reserved", c_int32),
                ("cameras", ctypes.POINTER(gs_camera)), ("pair_capacity", c_int64),
                ("record_capacity", c_int64)]


class gs_schedule(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("sub_buckets", c_int32), ("fwd_batch", c_int32),
                ("bwd_batch", c_int32), ("flags", c_int32)]


GS_SCHED_FUSED = 1  # gs_track_step: forward, fused loss and pose-only reverse walk in one kernel per tile
GS_SCHED_RADIX = 2  # the depth order from one device-wide LSD radix sort of the (tile, depth) keys


def radix_passes(tiles: int) -> int:
    """Eight-bit passes of the radix sort over `tiles` tiles: four for the depth bits and
    one per byte of the largest tile index."""
    bits = max(0, int(tiles - 1).bit_length())
    return 4 + (bits + 7) // 8


class gs_tune_entry(ctypes.Structure):
    _fields_ = [("stage", c_int32), ("ms", ctypes.c_float), ("schedule", gs_schedule)]


SCHEDULE_FIELDS = ("tile_w", "tile_h", "sub_buckets", "fwd_batch", "bwd_batch", "flags")


def schedule_dict(s: gs_schedule) -> dict:
    return {k: int(getattr(s, k)) for k in SCHEDULE_FIELDS}


class gs_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("ms", ctypes.c_float)]


class gs_counts(ctypes.Structure):
    _fields_ = [("n_records", c_int64), ("n_pairs", c_int64), ("err_flags", c_uint32), ("reserved", c_uint32),
                ("fwd_evals", c_int64), ("fwd_contrib", c_int64), ("bwd_evals", c_int64), ("bwd_contrib", c_int64),
                ("max_tile", c_uint32), ("reserved2", c_uint32)]


_lib = None
_lib_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgsgb.so (building it first if it is missing or stale).  Raises if no CUDA
    device is available: the rasterizer has no host fallback."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2408_05635_gb300 needs a CUDA GPU (sm_103a); none is available")
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        sigs = {
            "gs_default_config": (None, [P(gs_config)]),
            "gs_create": (c_int32, [P(c_void_p), P(gs_config)]),
            "gs_destroy": (c_int32, [c_void_p]),
            "gs_last_error": (ctypes.c_char_p, [c_void_p]),
            "gs_status_string": (ctypes.c_char_p, [c_int32]),
            "gs_workspace_size": (c_int32, [c_void_p, P(gs_problem), P(c_size_t)]),
            "gs_project": (c_int32, [c_void_p, P(gs_problem), P(gs_gaussians), c_void_p, c_void_p, c_size_t,
                                     c_void_p]),
            "gs_forward": (c_int32, [c_void_p, P(gs_targets), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
            "gs_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, P(gs_gaussians_grad), c_void_p,
                                      c_void_p]),
            "gs_track_step": (c_int32, [c_void_p, P(gs_problem), P(gs_gaussians), P(gs_targets), c_void_p,
                                        c_void_p, c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
            "gs_track_step_upload": (c_int32, [c_void_p, P(gs_problem), P(gs_gaussians), P(gs_targets),
                                               P(gs_host_targets), c_void_p, c_void_p, c_void_p, c_int32, c_void_p,
                                               c_size_t, c_void_p]),
            "gs_sync_status": (c_int32, [c_void_p, c_void_p, P(gs_counts)]),
            "gs_set_profiling": (c_int32, [c_void_p, c_int32]),
            "gs_set_profiling_mask": (c_int32, [c_void_p, ctypes.c_uint32]),
            "gs_render_static": (c_int32, [P(gs_config), P(gs_gaussians), P(gs_camera), c_void_p, P(gs_targets),
                                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
            "gs_kernel_times": (c_int32, [c_void_p, P(gs_kernel_time), c_int32, P(c_int32)]),
            "gs_get_schedule": (c_int32, [c_void_p, P(gs_schedule)]),
            "gs_pose_partials": (c_int32, [c_void_p, c_void_p, c_int64, P(c_int64), c_void_p]),
            "gs_set_schedule": (c_int32, [c_void_p, P(gs_schedule)]),
            "gs_autotune": (c_int32, [c_void_p, P(gs_problem), P(gs_gaussians), c_void_p, P(gs_targets), c_int32,
                                      c_int32, c_void_p, c_size_t, P(gs_tune_entry), c_int32, P(c_int32),
                                      P(gs_schedule), c_void_p]),
            "gs_image_metrics": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
            "gs_msssim_scratch_bytes": (c_size_t, [c_int32, c_int32]),
            "gs_msssim": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_size_t, c_void_p]),
            "gs_default_map_config": (None, [P(gs_map_config)]),
            "gs_map_scratch_bytes": (c_size_t, [c_int64]),
            "gs_map_add": (c_int32, [P(gs_map_config), P(gs_map), c_void_p, P(gs_camera), c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
            "gs_map_adam_step": (c_int32, [P(gs_map_config), P(gs_map), c_void_p, P(gs_gaussians_grad), c_int64,
                                           c_void_p]),
            "gs_map_prune": (c_int32, [P(gs_map_config), P(gs_map), c_void_p, P(gs_map), c_void_p, c_void_p,
                                       c_size_t, c_void_p]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class GsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ----------------------------------------------------------------------------- raw C names

def gs_default_config() -> gs_config:
    c = gs_config()
    load().gs_default_config(ctypes.byref(c))
    return c


def gs_create(cfg: gs_config | None = None) -> int:
    h = c_void_p()
    st = load().gs_create(ctypes.byref(h), ctypes.byref(cfg) if cfg is not None else None)
    if st:
        raise GsError(st, "gs_create")
    return h.value


def gs_destroy(ctx: int) -> None:
    load().gs_destroy(ctx)


def gs_last_error(ctx: int) -> str:
    return (load().gs_last_error(ctx) or b"").decode()


def _check(ctx, st, what):
    if st:
        raise GsError(st, f"{what}: {gs_last_error(ctx)}")


def gs_workspace_size(ctx: int, prob: gs_problem) -> int:
    n = c_size_t(0)
    _check(ctx, load().gs_workspace_size(ctx, ctypes.byref(prob), ctypes.byref(n)), "gs_workspace_size")
    return n.value


def gs_project(ctx, prob: gs_problem, g: gs_gaussians, poses: torch.Tensor, ws: torch.Tensor, ws_bytes: int,
               stream=None) -> None:
    _check(ctx, load().gs_project(ctx, ctypes.byref(prob), ctypes.byref(g), _ptr(poses), _ptr(ws), ws_bytes,
                                  _stream(stream)), "gs_project")


def gs_forward(ctx, targets: gs_targets | None, rgb=None, depth=None, sil=None, loss=None, stream=None) -> None:
    _check(ctx, load().gs_forward(ctx, ctypes.byref(targets) if targets is not None else None, _ptr(rgb),
                                  _ptr(depth), _ptr(sil), _ptr(loss), _stream(stream)), "gs_forward")


def gs_backward(ctx, d_rgb=None, d_depth=None, d_sil=None, grads: gs_gaussians_grad | None = None,
                pose_grad=None, stream=None) -> None:
    _check(ctx, load().gs_backward(ctx, _ptr(d_rgb), _ptr(d_depth), _ptr(d_sil),
                                   ctypes.byref(grads) if grads is not None else None, _ptr(pose_grad),
                                   _stream(stream)), "gs_backward")


def gs_track_step(ctx, prob: gs_problem, g: gs_gaussians, targets: gs_targets, poses, adam_state, loss_hist,
                  iters: int, ws, ws_bytes: int, stream=None) -> None:
    _check(ctx, load().gs_track_step(ctx, ctypes.byref(prob), ctypes.byref(g), ctypes.byref(targets), _ptr(poses),
                                     _ptr(adam_state), _ptr(loss_hist), int(iters), _ptr(ws), ws_bytes,
                                     _stream(stream)), "gs_track_step")


def gs_track_step_upload(ctx, prob: gs_problem, g: gs_gaussians, targets, src: gs_host_targets, poses,
                         adam_state, loss_hist, iters: int, ws, ws_bytes: int, stream=None) -> None:
    """gs_track_step with the frame in page-locked host memory (src): copied into the
    device targets beside the first iteration's binning, or, with targets None, read in
    place by the kernels."""
    _check(ctx, load().gs_track_step_upload(ctx, ctypes.byref(prob), ctypes.byref(g),
                                            ctypes.byref(targets) if targets is not None else None,
                                            ctypes.byref(src), _ptr(poses), _ptr(adam_state), _ptr(loss_hist),
                                            int(iters), _ptr(ws), ws_bytes, _stream(stream)), "gs_track_step_upload")


def gs_sync_status(ctx, stream=None) -> tuple[int, gs_counts]:
    """Returns (status, counts); status GS_ERR_CAPACITY / GS_ERR_TIMEOUT are not raised."""
    c = gs_counts()
    st = load().gs_sync_status(ctx, _stream(stream), ctypes.byref(c))
    if st not in (0, GS_ERR_CAPACITY, 6):
        raise GsError(st, f"gs_sync_status: {gs_last_error(ctx)}")
    return st, c


def gs_set_profiling(ctx, enable: bool) -> None:
    _check(ctx, load().gs_set_profiling(ctx, int(bool(enable))), "gs_set_profiling")


KERNELS = ("k_project", "k_scan_tiles", "k_emit", "k_forward", "k_backward", "k_bproject", "k_finalize",
           "k_track_tile", "k_radix_sort")


def gs_set_profiling_mask(ctx, kernels) -> None:
    """Bracket only the named kernels (names from KERNELS) with profiling markers."""
    mask = 0
    for k in kernels:
        mask |= 1 << KERNELS.index(k)
    _check(ctx, load().gs_set_profiling_mask(ctx, mask), "gs_set_profiling_mask")


def gs_kernel_times(ctx, cap: int = 4096) -> list[tuple[str, float]]:
    """(kernel name, ms) of every library kernel of the last enqueued sequence."""
    arr = (gs_kernel_time * cap)()
    cnt = c_int32(0)
    _check(ctx, load().gs_kernel_times(ctx, arr, cap, ctypes.byref(cnt)), "gs_kernel_times")
    return [(arr[k].name.decode(), float(arr[k].ms)) for k in range(min(cap, cnt.value))]


def gs_pose_partials(ctx, stream=None) -> np.ndarray:
    """The per-cell double-float pose partials of the last pose backward: an array of
    shape (views, cells, 6, 2) of (hi, lo) FP32 pairs."""
    cnt = c_int64(0)
    _check(ctx, load().gs_pose_partials(ctx, None, 0, ctypes.byref(cnt), _stream(stream)), "gs_pose_partials")
    out = np.zeros(cnt.value, dtype=np.float32)
    _check(ctx, load().gs_pose_partials(ctx, out.ctypes.data, cnt.value, ctypes.byref(cnt), _stream(stream)),
           "gs_pose_partials")
    return out.reshape(-1, 6, 2)


def gs_get_schedule(ctx) -> gs_schedule:
    s = gs_schedule()
    _check(ctx, load().gs_get_schedule(ctx, ctypes.byref(s)), "gs_get_schedule")
    return s


def gs_set_schedule(ctx, tile_w: int, tile_h: int, sub_buckets: int, fwd_batch: int, bwd_batch: int,
                    flags: int = 0) -> None:
    s = gs_schedule(int(tile_w), int(tile_h), int(sub_buckets), int(fwd_batch), int(bwd_batch), int(flags))
    _check(ctx, load().gs_set_schedule(ctx, ctypes.byref(s)), "gs_set_schedule")


TUNE_STAGES = ("tile", "sub_buckets", "fwd_batch", "bwd_batch", "fused", "sort")
TUNE_MAX = 17


def gs_autotune(ctx, prob: gs_problem, g: gs_gaussians, poses, targets: gs_targets, ws, ws_bytes: int,
                pose_only: bool = True, reps: int = 10, stream=None) -> tuple[gs_schedule, list[tuple[str, dict, float]]]:
    """Time the tile shapes, sub-bucket counts and batch depths on this problem, set the
    fastest on the context and return it with the measurements (stage, schedule timed,
    ms per pass; -1 where the setting overflowed the pair capacity)."""
    table = (gs_tune_entry * TUNE_MAX)()
    cnt = c_int32(0)
    best = gs_schedule()
    st = load().gs_autotune(ctx, ctypes.byref(prob), ctypes.byref(g), _ptr(poses), ctypes.byref(targets),
                            int(bool(pose_only)), int(reps), _ptr(ws), ws_bytes, table, TUNE_MAX,
                            ctypes.byref(cnt), ctypes.byref(best), _stream(stream))
    _check(ctx, st, "gs_autotune")
    rows = [(TUNE_STAGES[table[k].stage], schedule_dict(table[k].schedule), float(table[k].ms))
            for k in range(min(TUNE_MAX, cnt.value))]
    return best, rows


def gs_render_static(cfg: gs_config, g: gs_gaussians, cam: gs_camera, pose, targets: gs_targets | None = None,
                     rgb=None, depth=None, sil=None, loss=None, err_flags=None, stream=None) -> None:
    """Single-view render whose scratch is a static device array of the library: no
    workspace, no allocation (see include/gs.h for the limits and the sharing rules)."""
    st = load().gs_render_static(ctypes.byref(cfg), ctypes.byref(g), ctypes.byref(cam), _ptr(pose),
                                 ctypes.byref(targets) if targets is not None else None, _ptr(rgb), _ptr(depth),
                                 _ptr(sil), _ptr(loss), _ptr(err_flags), _stream(stream))
    if st:
        raise GsError(st, "gs_render_static")


# ----------------------------------------------------------------------------- convenience

@dataclasses.dataclass
class Config:
    """Python mirror of gs_config (defaults = gs_default_config)."""
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    dilation: float = 0.0
    z_near: float = 0.2
    jac_clip: float = 1.3
    sil_thresh: float = 0.99
    w_rgb: float = 0.5
    w_depth: float = 1.0
    w_vis: float = 0.1
    w_prior: float = 0.5
    lr_rot: float = 2e-3
    lr_trans: float = 2e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def c(self) -> gs_config:
        g = gs_config()
        g.tile_w = g.tile_h = 16
        for f in dataclasses.fields(self):
            setattr(g, f.name, getattr(self, f.name))
        return g


_DT = {torch.float32: GS_F32, torch.bfloat16: GS_BF16, torch.float16: GS_F16}


@dataclasses.dataclass
class GaussianTensors:
    """Device tensors of a Gaussian map: means float32 n x 3; quats n x 4; log_scales
    n x 3; logits n; rgb n x 3 (the last four share one dtype: float32, bfloat16 or
    float16)."""
    means: torch.Tensor
    quats: torch.Tensor
    log_scales: torch.Tensor
    logits: torch.Tensor
    rgb: torch.Tensor

    @property
    def n(self) -> int:
        return self.means.shape[0]

    @property
    def isotropic(self) -> bool:
        """Eq. 1 as written: no quaternions, one log-radius per Gaussian."""
        return self.quats is None

    def c(self) -> gs_gaussians:
        if self.means.dtype != torch.float32:
            raise ValueError("means must be float32")
        dt = self.log_scales.dtype
        for t in (self.logits, self.rgb) + (() if self.quats is None else (self.quats,)):
            if t.dtype != dt:
                raise ValueError("quats, log_scales, logits and rgb must share one dtype")
        if dt not in _DT:
            raise ValueError(f"unsupported attribute dtype {dt}")
        if self.quats is None and self.log_scales.numel() != self.n:
            raise ValueError("isotropic Gaussians take one log-radius each")
        return gs_gaussians(_ptr(self.means), _ptr(self.quats), _ptr(self.log_scales), _ptr(self.logits),
                            _ptr(self.rgb), _DT[dt], 0, self.n)

    @staticmethod
    def from_numpy(g, device="cuda", attr_dtype=torch.float32) -> "GaussianTensors":
        def t(a, dt):
            return torch.as_tensor(a, dtype=torch.float32).to(device=device, dtype=dt).contiguous()
        return GaussianTensors(t(g.means, torch.float32), None if g.quats is None else t(g.quats, attr_dtype),
                               t(g.log_scales, attr_dtype), t(g.logits, attr_dtype), t(g.rgb, attr_dtype))


def gs_image_metrics(rgb, depth, rgb_t, depth_t, out: torch.Tensor, stream=None) -> None:
    """out (device, 4 doubles) <- (sum sq. colour error, sum |D - D*| where D* > 0, that
    pixel count, sum (D - D*)^2 there)."""
    _map_check(load().gs_image_metrics(_ptr(rgb), _ptr(depth), _ptr(rgb_t), _ptr(depth_t), int(depth.numel()), _ptr(out),
                                       _stream(stream)), "gs_image_metrics")


def gs_msssim(rgb, rgb_t, width: int, height: int, out: torch.Tensor, stream=None) -> None:
    """out (device, 4 doubles) <- MS-SSIM (channel mean, red, green, blue) of two planar
    colour images; the scratch is allocated here."""
    need = int(load().gs_msssim_scratch_bytes(int(width), int(height)))
    scratch = torch.empty(need + 256, dtype=torch.uint8, device=out.device)
    off = (-scratch.data_ptr()) % 256
    _map_check(load().gs_msssim(_ptr(rgb), _ptr(rgb_t), int(width), int(height), _ptr(out),
                                scratch[off:].data_ptr(), need, _stream(stream)), "gs_msssim")


def gs_default_map_config() -> gs_map_config:
    c = gs_map_config()
    load().gs_default_map_config(ctypes.byref(c))
    return c


def gs_map_scratch_bytes(items: int) -> int:
    return int(load().gs_map_scratch_bytes(int(items)))


def _map_check(st, what):
    if st:
        raise GsError(st, what)


def gs_map_add(cfg: gs_map_config, m: gs_map, n: torch.Tensor, cam, pose: torch.Tensor, rgb, depth, sil, scratch,
               scratch_bytes: int, err=None, stream=None) -> None:
    _map_check(load().gs_map_add(ctypes.byref(cfg), ctypes.byref(m), _ptr(n), ctypes.byref(cam), _ptr(pose), _ptr(rgb),
                                 _ptr(depth), _ptr(sil), _ptr(scratch), scratch_bytes, _ptr(err), _stream(stream)),
               "gs_map_add")


def gs_map_adam_step(cfg: gs_map_config, m: gs_map, n: torch.Tensor, grads: gs_gaussians_grad, step: int,
                     stream=None) -> None:
    _map_check(load().gs_map_adam_step(ctypes.byref(cfg), ctypes.byref(m), _ptr(n), ctypes.byref(grads), int(step),
                                       _stream(stream)), "gs_map_adam_step")


def gs_map_prune(cfg: gs_map_config, src: gs_map, n_src: torch.Tensor, dst: gs_map, n_dst: torch.Tensor, scratch,
                 scratch_bytes: int, stream=None) -> None:
    _map_check(load().gs_map_prune(ctypes.byref(cfg), ctypes.byref(src), _ptr(n_src), ctypes.byref(dst), _ptr(n_dst),
                                   _ptr(scratch), scratch_bytes, _stream(stream)), "gs_map_prune")


class Map:
    """The map as the scene optimisation holds it (gs_map): FP32 master arrays with room
    for `capacity` Gaussians (rounded up to a multiple of 4), the live count on the device,
    the Adam moments and, with lowp_dtype, a BF16 / F16 render copy of the attributes.
    isotropic: Eq. 1 as written (no quaternions, one log-radius per Gaussian)."""

    def __init__(self, capacity: int, device="cuda", lowp_dtype: torch.dtype | None = None, adam: bool = True,
                 config: gs_map_config | None = None, isotropic: bool = False):
        load()
        cap = (int(capacity) + 3) // 4 * 4
        self.capacity, self.device, self.isotropic = cap, torch.device(device), isotropic
        self.GROUPS = ("means", "log_scales", "logits", "rgb") if isotropic else ("means", "quats", "log_scales",
                                                                                  "logits", "rgb")
        self.WIDTH = {"means": 3, "quats": 4, "log_scales": 1 if isotropic else 3, "logits": 1, "rgb": 3}
        self.p = {k: torch.zeros((cap, self.WIDTH[k]) if k != "logits" else (cap,), dtype=torch.float32, device=device)
                  for k in self.GROUPS}
        self.lowp_dtype = lowp_dtype
        self.lp = None if lowp_dtype is None else {
            k: torch.zeros_like(self.p[k], dtype=lowp_dtype) for k in self.GROUPS if k != "means"}
        per = sum(self.WIDTH[k] for k in self.GROUPS)
        self.state = torch.zeros(2 * per * cap, dtype=torch.float32, device=device) if adam else None
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.err = torch.zeros(1, dtype=torch.int32, device=device)
        self.config = config or gs_default_map_config()
        self._scratch = None

    def c(self) -> gs_map:
        lp = self.lp or {}
        return gs_map(_ptr(self.p["means"]), _ptr(self.p.get("quats")), _ptr(self.p["log_scales"]), _ptr(self.p["logits"]),
                      _ptr(self.p["rgb"]), _ptr(lp.get("quats")), _ptr(lp.get("log_scales")), _ptr(lp.get("logits")),
                      _ptr(lp.get("rgb")), _DT.get(self.lowp_dtype, 0), 0, self.capacity, _ptr(self.state))

    @property
    def n(self) -> int:
        """Live count (synchronises with the device)."""
        return int(self.count.item())

    def scratch(self, items: int) -> tuple[torch.Tensor, int]:
        need = gs_map_scratch_bytes(items)
        if self._scratch is None or self._scratch.numel() < need + 256:
            self._scratch = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        off = (-self._scratch.data_ptr()) % 256
        return self._scratch[off:off + need], need

    def gaussians(self, n: int | None = None, lowp: bool = False) -> GaussianTensors:
        """The first n live Gaussians as a render input (FP32, or the low-precision copy)."""
        n = self.n if n is None else n
        src = self.lp if lowp else self.p
        q = None if self.isotropic else src["quats"][:n]
        return GaussianTensors(self.p["means"][:n], q, src["log_scales"][:n], src["logits"][:n], src["rgb"][:n])

    def load(self, g) -> None:
        """Fill the map with arrays (numpy or tensors, rows = Gaussians); moments zeroed."""
        n = len(g.means)
        if n > self.capacity:
            raise ValueError("more Gaussians than capacity")
        for k in self.GROUPS:
            a = torch.as_tensor(getattr(g, k), dtype=torch.float32, device=self.device)
            if k == "log_scales" and self.isotropic and a.dim() == 2 and a.shape[1] == 3:
                a = a.mean(dim=1)
            self.p[k][:n] = a.reshape(self.p[k][:n].shape)
            if self.lp is not None and k != "means":
                self.lp[k][:n] = self.p[k][:n].to(self.lowp_dtype)
        if self.state is not None:
            self.state.zero_()
        self.count.fill_(n)

    def add_from_frame(self, cam, pose: torch.Tensor, rgb, depth, sil=None, stream=None) -> None:
        """gs_map_add: Gaussians for the frame's pixels with depth (and S < sil_add)."""
        cc = gs_camera(float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy), int(cam.width), int(cam.height))
        scr, nb = self.scratch(int(cam.width) * int(cam.height))
        gs_map_add(self.config, self.c(), self.count, cc, pose, rgb, depth, sil, scr, nb, self.err, stream)

    def adam_step(self, grads: dict, step: int, stream=None) -> None:
        """gs_map_adam_step with gradient tensors of capacity rows (keys of GROUPS)."""
        G = gs_gaussians_grad(_ptr(grads.get("means")), _ptr(grads.get("quats")), _ptr(grads.get("log_scales")),
                              _ptr(grads.get("logits")), _ptr(grads.get("rgb")))
        gs_map_adam_step(self.config, self.c(), self.count, G, step, stream)

    def prune_into(self, dst: "Map", stream=None) -> None:
        """gs_map_prune: the Gaussians of this map with opacity >= opacity_min, into dst."""
        scr, nb = self.scratch(self.capacity)
        gs_map_prune(self.config, self.c(), self.count, dst.c(), dst.count, scr, nb, stream)


def cameras_c(cams: Sequence) -> ctypes.Array:
    arr = (gs_camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = gs_camera(float(c.fx), float(c.fy), float(c.cx), float(c.cy), int(c.width), int(c.height))
    return arr


class Rasterizer:
    """Owns a context and a workspace; marshals torch tensors into the C calls."""

    def __init__(self, config: Config | None = None, device: str | torch.device = "cuda"):
        load()
        self.config = config or Config()
        self.device = torch.device(device)
        self.ctx = gs_create(self.config.c())
        self._ws = None
        self._ws_view = None
        self._keep = []

    def close(self):
        if getattr(self, "ctx", None):
            gs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- workspace ---------------------------------------------------------------------
    def problem(self, n: int, cams: Sequence, pair_capacity: int) -> gs_problem:
        arr = cameras_c(cams)
        p = gs_problem(int(n), len(cams), 0, ctypes.cast(arr, ctypes.POINTER(gs_camera)), int(pair_capacity), 0)
        p._cams = arr  # keep the host array alive with the struct
        return p

    def workspace(self, prob: gs_problem) -> tuple[torch.Tensor, int]:
        need = gs_workspace_size(self.ctx, prob)
        if self._ws is None or self._ws.numel() < need + 256:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        off = (-self._ws.data_ptr()) % 256
        view = self._ws[off:off + need]
        return view, need

    def measure(self, g: GaussianTensors, cams: Sequence, poses: torch.Tensor) -> tuple[int, int]:
        """Project once with minimal capacities and return (pairs, records) of the scene."""
        prob = self.problem(g.n, cams, pair_capacity=1)
        ws, nb = self.workspace(prob)
        gs_project(self.ctx, prob, g.c(), poses, ws, nb)
        _, counts = gs_sync_status(self.ctx)
        return int(counts.n_pairs), int(counts.n_records)

    def plan(self, g: GaussianTensors, cams: Sequence, poses: torch.Tensor, margin: float = 1.25,
             min_pairs: int = 1024) -> gs_problem:
        pairs, _ = self.measure(g, cams, poses)
        return self.problem(g.n, cams, max(min_pairs, int(pairs * margin) + 1024))

    # -- one rendering pass ------------------------------------------------------------
    def render(self, prob: gs_problem, g: GaussianTensors, poses: torch.Tensor, targets=None, stream=None,
               images: bool = True) -> dict:
        """gs_project + gs_forward.  targets = (rgb, depth, prior-or-None) tensors enable
        the fused loss.  Returns the images (and loss) as tensors."""
        ws, nb = self.workspace(prob)
        gs_project(self.ctx, prob, g.c(), poses, ws, nb, stream)
        P = sum(int(c.width) * int(c.height) for c in prob._cams)
        out = {}
        if images:
            out["rgb"] = torch.empty(3 * P, device=self.device)
            out["depth"] = torch.empty(P, device=self.device)
            out["sil"] = torch.empty(P, device=self.device)
        tg = None
        if targets is not None:
            trgb, tdep, tprior = targets
            tg = gs_targets(_ptr(trgb), _ptr(tdep), _ptr(tprior))
            out["loss"] = torch.empty(prob.n_views, dtype=torch.float64, device=self.device)
        gs_forward(self.ctx, tg, out.get("rgb"), out.get("depth"), out.get("sil"), out.get("loss"), stream)
        self._keep = [g, poses, targets]
        return out

    def backward(self, g: GaussianTensors, upstream=None, params: bool = True, pose: bool = True,
                 stream=None, n_views: int = 1) -> dict:
        out = {}
        grads = None
        if params:
            out["grads"] = {k: torch.zeros(getattr(g, k).shape, dtype=torch.float32, device=self.device)
                            for k in ("means", "quats", "log_scales", "logits", "rgb") if getattr(g, k) is not None}
            G = out["grads"]
            grads = gs_gaussians_grad(_ptr(G["means"]), _ptr(G.get("quats")), _ptr(G["log_scales"]), _ptr(G["logits"]),
                                      _ptr(G["rgb"]))
        if pose:
            out["pose_grad"] = torch.zeros(n_views, 6, dtype=torch.float64, device=self.device)
        up = upstream if upstream is not None else (None, None, None)
        gs_backward(self.ctx, up[0], up[1], up[2], grads, out.get("pose_grad"), stream)
        return out

    def mapping_grads(self, g: GaussianTensors, cams: Sequence, poses: torch.Tensor, targets: Sequence,
                      chunk: int = 2, grads: dict | None = None, probs: list | None = None, stream=None) -> dict:
        """Gradients of the combined loss summed over a keyframe window (Sec. III-C: poses
        fixed, Gaussians updated).  Views are processed `chunk` at a time through one
        workspace: each chunk is projected, binned, sorted, composited and differentiated
        before the next, so the per-tile lists and transmittances of the window are
        recomputed per chunk and never stored together.  targets: per view (rgb 3HW,
        depth HW, prior HW or None) device tensors.  Returns {'grads': ..., 'loss': V}."""
        V = len(cams)
        if grads is None:
            grads = {k: torch.zeros(getattr(g, k).shape, dtype=torch.float32, device=self.device)
                     for k in ("means", "quats", "log_scales", "logits", "rgb") if getattr(g, k) is not None}
        G = gs_gaussians_grad(_ptr(grads["means"]), _ptr(grads.get("quats")), _ptr(grads["log_scales"]),
                              _ptr(grads["logits"]), _ptr(grads["rgb"]))
        loss = torch.zeros(V, dtype=torch.float64, device=self.device)
        gc = g.c()
        for ci, v0 in enumerate(range(0, V, chunk)):
            sl = slice(v0, min(V, v0 + chunk))
            vc = list(cams[sl])
            prob = probs[ci] if probs is not None else self.plan(g, vc, poses[sl].contiguous())
            ws, nb = self.workspace(prob)
            tg = targets[sl]
            t_rgb = torch.cat([t[0].reshape(-1) for t in tg]).contiguous()
            t_depth = torch.cat([t[1].reshape(-1) for t in tg]).contiguous()
            has_prior = all(t[2] is not None for t in tg)
            t_prior = torch.cat([t[2].reshape(-1) for t in tg]).contiguous() if has_prior else None
            self._keep = [t_rgb, t_depth, t_prior]
            gs_project(self.ctx, prob, gc, poses[sl].contiguous(), ws, nb, stream)
            gs_forward(self.ctx, gs_targets(_ptr(t_rgb), _ptr(t_depth), _ptr(t_prior)), None, None, None,
                       loss[sl], stream)
            gs_backward(self.ctx, None, None, None, G, None, stream)
        return {"grads": grads, "loss": loss}

    # -- launch schedule -----------------------------------------------------------------
    @property
    def schedule(self) -> dict:
        return schedule_dict(gs_get_schedule(self.ctx))

    def set_schedule(self, tile_w: int = 16, tile_h: int = 16, sub_buckets: int = 4, fwd_batch: int = 256,
                     bwd_batch: int = 256, flags: int = 0) -> None:
        gs_set_schedule(self.ctx, tile_w, tile_h, sub_buckets, fwd_batch, bwd_batch, flags)

    def autotune(self, prob: gs_problem, g: GaussianTensors, poses: torch.Tensor, targets, pose_only: bool = True,
                 reps: int = 10, stream=None) -> dict:
        """gs_autotune on this problem; targets = (rgb, depth, prior-or-None) tensors
        concatenated over the views.  Returns the chosen schedule and the timings."""
        ws, nb = self.workspace(prob)
        trgb, tdep, tprior = targets
        tg = gs_targets(_ptr(trgb), _ptr(tdep), _ptr(tprior))
        best, rows = gs_autotune(self.ctx, prob, g.c(), poses, tg, ws, nb, pose_only, reps, stream)
        return {"schedule": schedule_dict(best),
                "timings_ms": [{"stage": k, "schedule": sc, "ms": round(ms, 4)} for k, sc, ms in rows]}

    def sync(self, stream=None) -> gs_counts:
        st, c = gs_sync_status(self.ctx, stream)
        if st:
            raise GsError(st, gs_last_error(self.ctx))
        return c
