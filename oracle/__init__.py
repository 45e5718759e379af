"""FP64 CPU oracle for the differentiable 3D-Gaussian rasterizer (arXiv 2408.05635).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA product path never does.
It shares no code with the CUDA library (``paper_2408_05635_gb300``).

The arithmetic lives in ``gs_oracle.c`` (plain C, FP64, OpenMP over pixel rows); this
module only compiles it, marshals numpy arrays through ctypes and returns numpy arrays.
Every function documents the paper passage it follows; see the C file's header for the
readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Camera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class _Params(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in (
        "alpha_min", "alpha_max", "t_min", "dilation", "z_near", "jac_clip", "sil_thresh",
        "w_rgb", "w_depth", "w_vis", "w_prior", "beta1", "beta2", "eps", "lr_rot", "lr_trans",
        "amb_alpha", "amb_t", "amb_sil", "amb_resid", "amb_effect")] + [
        ("brute_force", ctypes.c_int32), ("n_threads", ctypes.c_int32)]


class _Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64)] + [(name, ctypes.POINTER(ctypes.c_double)) for name in (
        "means", "quats", "log_scales", "logits", "rgb")]


@dataclasses.dataclass
class Params:
    """Renderer, loss and optimiser settings (the readings listed in gs_oracle.c).

    alpha_max / alpha_min / t_min: opacity clamp, skip threshold and early-termination
    transmittance; z_near: near plane (m); dilation: eps added to Sigma' (px^2);
    jac_clip: the Jacobian of Sigma' is taken at the mean's image-plane tangent clamped
    to +-jac_clip half-extents of the view (0 disables the clamp);
    sil_thresh and the w_* weights define the combined loss; beta1/beta2/eps/lr_* the
    decoupled Adam; amb_* the floors of the ambiguity-mask margins (which otherwise follow
    the FP32 error of the footprint exponent at each pixel), amb_effect the smallest pixel
    change an alpha_min decision must be able to make to count; brute_force selects the
    walk over every Gaussian instead of the opacity-aware boxes.
    """
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
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    lr_rot: float = 2e-3
    lr_trans: float = 2e-3
    amb_alpha: float = 2e-4
    amb_t: float = 2e-4
    amb_sil: float = 1e-5
    amb_resid: float = 2e-5
    amb_effect: float = 2.5e-5
    brute_force: bool = False
    n_threads: int = 0

    def _c(self) -> _Params:
        p = _Params()
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            setattr(p, f.name, int(v) if f.name in ("brute_force", "n_threads") else float(v))
        return p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            d, i64, i32, u8 = (P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_int32),
                               P(ctypes.c_uint8))
            sc, cam, par = P(_Scene), P(Camera), P(_Params)
            lib.og_project.argtypes = [sc, cam, d, par, d]
            lib.og_render.argtypes = [sc, cam, d, par, d, d, d, d, i32, u8]
            lib.og_render_pixels.argtypes = [sc, cam, d, par, i64, ctypes.c_int64, d, d, u8]
            lib.og_loss.argtypes = [cam, par, d, d, d, d, d, d, d, d, d, d, u8]
            lib.og_backward.argtypes = [sc, cam, d, par, d, d, d, d, d, d]
            lib.og_adam_step.argtypes = [d, d, d, par]
            lib.og_num_threads.argtypes = [par]
            lib.og_render_perturbed.argtypes = [sc, cam, d, par, ctypes.c_uint64, ctypes.c_double, ctypes.c_int32, d, d, d, d]
            lib.og_render_alternatives.argtypes = [sc, cam, d, par, i64, ctypes.c_int64, ctypes.c_int32, i32, d]
            lib.og_depth_keys.argtypes = [sc, d, P(ctypes.c_float), d]
            lib.og_render_tstats.argtypes = [sc, cam, d, par, d, d]
            for fn in (lib.og_project, lib.og_render, lib.og_render_pixels, lib.og_loss,
                       lib.og_backward, lib.og_adam_step, lib.og_num_threads, lib.og_render_perturbed,
                       lib.og_render_alternatives, lib.og_depth_keys, lib.og_render_tstats):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


class Scene:
    """FP64 copy of a Gaussian map (means n x 3, quats n x 4 (w,x,y,z), log_scales n x 3,
    opacity logits n, rgb n x 3).  The parameters of Eq. 1 in their anisotropic form."""

    def __init__(self, means, quats, log_scales, logits, rgb):
        self.means = _f64(means).reshape(-1, 3)
        n = self.means.shape[0]
        self.quats = _f64(quats, (n, 4))
        self.log_scales = _f64(log_scales, (n, 3))
        self.logits = _f64(logits, (n,))
        self.rgb = _f64(rgb, (n, 3))
        self.n = n

    def _c(self) -> _Scene:
        s = _Scene()
        s.n = self.n
        s.means, s.quats, s.log_scales, s.logits, s.rgb = (
            _dp(self.means), _dp(self.quats), _dp(self.log_scales), _dp(self.logits), _dp(self.rgb))
        return s


def camera(fx, fy, cx, cy, width, height) -> Camera:
    """Pinhole intrinsics of pi_m (Sec. II-A) and the image size in pixels."""
    return Camera(float(fx), float(fy), float(cx), float(cy), int(width), int(height))


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def project(scene: Scene, cam: Camera, pose, params: Params) -> dict:
    """Per-Gaussian projection (Sec. II-A pi_m; Sigma' = J W Sigma W^T J^T of Sec. I).

    Returns arrays: valid, mu (n x 2), z, cov2 (A, B, C), conic (a, b, c), opacity,
    dmax2 (opacity-aware squared Mahalanobis support), box (x0, x1, y0, y1)."""
    lib = _load()
    out = np.zeros((scene.n, 16))
    sc, par, pose = scene._c(), params._c(), _f64(pose, (7,))
    _check(lib.og_project(ctypes.byref(sc), ctypes.byref(cam), _dp(pose), ctypes.byref(par), _dp(out)),
           "project")
    return {"valid": out[:, 0] > 0.5, "mu": out[:, 1:3], "z": out[:, 3], "cov2": out[:, 4:7],
            "conic": out[:, 7:10], "opacity": out[:, 10], "dmax2": out[:, 11],
            "box": out[:, 12:16].astype(np.int64)}


def render(scene: Scene, cam: Camera, pose, params: Params) -> dict:
    """Eqs. 2-4: colour (3 x H x W), depth and silhouette (H x W), final transmittance,
    number of contributors and the ambiguity mask, every pixel.  amb_bits holds the
    reasons a pixel is flagged: AMB_ALPHA_MIN (an alpha near alpha_min whose skip matters),
    AMB_ALPHA_MAX (an alpha near the clamp; it changes gradients, not the maps) and
    AMB_T_MIN (the transmittance reaches t_min within its margin)."""
    lib = _load()
    H, W = cam.height, cam.width
    rgb = np.zeros((3, H, W))
    depth = np.zeros((H, W))
    sil = np.zeros((H, W))
    tf = np.zeros((H, W))
    nc = np.zeros((H, W), dtype=np.int32)
    amb = np.zeros((H, W), dtype=np.uint8)
    sc, par, pose = scene._c(), params._c(), _f64(pose, (7,))
    _check(lib.og_render(ctypes.byref(sc), ctypes.byref(cam), _dp(pose), ctypes.byref(par), _dp(rgb),
                         _dp(depth), _dp(sil), _dp(tf), nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         amb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "render")
    return {"rgb": rgb, "depth": depth, "sil": sil, "t_final": tf, "n_contrib": nc, "amb": amb.astype(bool),
            "amb_bits": amb}


AMB_ALPHA_MIN, AMB_ALPHA_MAX, AMB_T_MIN = 1, 2, 4


def render_perturbed(scene: Scene, cam: Camera, pose, params: Params, seed: int, scale: float,
                     f32_pose: bool = False) -> dict:
    """A render within the FP32 error model the ambiguity mask assumes, for testing the
    mask: each screen mean moved by scale x up to dmu (the modelled camera-transform
    error) in a direction drawn per Gaussian, each (pixel, Gaussian) exponent of Eq. 1 by
    scale x up to its modelled rounding error (SplitMix64 uniforms from (seed, pixel,
    Gaussian)); with f32_pose, also the pose rounded to FP32 as the GPU applies it."""
    lib = _load()
    H, W = cam.height, cam.width
    rgb, depth, sil, tf = np.zeros((3, H, W)), np.zeros((H, W)), np.zeros((H, W)), np.zeros((H, W))
    sc, par, pose = scene._c(), params._c(), _f64(pose, (7,))
    _check(lib.og_render_perturbed(ctypes.byref(sc), ctypes.byref(cam), _dp(pose), ctypes.byref(par),
                                   ctypes.c_uint64(seed), float(scale), int(bool(f32_pose)), _dp(rgb), _dp(depth),
                                   _dp(sil), _dp(tf)),
           "render_perturbed")
    return {"rgb": rgb, "depth": depth, "sil": sil, "t_final": tf}


def render_alternatives(scene: Scene, cam: Camera, pose, params: Params, pix, max_alt: int = 16) -> dict:
    """Every outcome (C_r, C_g, C_b, D, S, T) an FP32 renderer may legitimately produce at
    the selected pixels (flat index y * W + x): the walk of Eqs. 2-4 branched at each
    decision the ambiguity mask flags.  n_alt[k] outcomes in alts[k, :n_alt[k]], or
    n_alt[k] = -1 when the pixel needs more than max_alt."""
    lib = _load()
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    n_alt = np.zeros(pix.size, dtype=np.int32)
    alts = np.zeros((pix.size, max_alt, 6))
    sc, par, pose = scene._c(), params._c(), _f64(pose, (7,))
    _check(lib.og_render_alternatives(ctypes.byref(sc), ctypes.byref(cam), _dp(pose), ctypes.byref(par),
                                      pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), pix.size, int(max_alt),
                                      n_alt.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(alts)),
           "render_alternatives")
    return {"n_alt": n_alt, "alts": alts}


def render_tstats(scene: Scene, cam: Camera, pose, params: Params) -> dict:
    """Per pixel, where the walk stops on t_min: the transmittance-error bound it carried
    (eT) and that step's size in log transmittance, -ln(1 - alpha) (0 where it does not
    stop)."""
    lib = _load()
    H, W = cam.height, cam.width
    eT, step = np.zeros((H, W)), np.zeros((H, W))
    sc, par, pose = scene._c(), params._c(), _f64(pose, (7,))
    _check(lib.og_render_tstats(ctypes.byref(sc), ctypes.byref(cam), _dp(pose), ctypes.byref(par), _dp(eT),
                                _dp(step)), "render_tstats")
    return {"eT": eT, "step": step}


def depth_keys(scene: Scene, pose) -> tuple[np.ndarray, np.ndarray]:
    """(FP32 depth key that orders Eqs. 2-4, FP64 camera-frame depth) of every Gaussian."""
    lib = _load()
    keys = np.zeros(scene.n, dtype=np.float32)
    z = np.zeros(scene.n)
    sc, pose = scene._c(), _f64(pose, (7,))
    _check(lib.og_depth_keys(ctypes.byref(sc), _dp(pose), keys.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             _dp(z)), "depth_keys")
    return keys, z


def render_pixels(scene: Scene, cam: Camera, pose, params: Params, pix) -> dict:
    """Eqs. 2-4 at selected pixels only (flat index y * W + x)."""
    lib = _load()
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    out = np.zeros((pix.size, 5))
    tf = np.zeros(pix.size)
    amb = np.zeros(pix.size, dtype=np.uint8)
    sc, par, pose = scene._c(), params._c(), _f64(pose, (7,))
    _check(lib.og_render_pixels(ctypes.byref(sc), ctypes.byref(cam), _dp(pose), ctypes.byref(par),
                                pix.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), pix.size, _dp(out), _dp(tf),
                                amb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), "render_pixels")
    return {"rgb": out[:, 0:3], "depth": out[:, 3], "sil": out[:, 4], "t_final": tf, "amb": amb.astype(bool)}


def loss(cam: Camera, params: Params, rgb, depth, sil, rgb_t, depth_t, prior=None) -> dict:
    """Combined loss of Sec. III-B (photometric + depth + visibility) plus the depth-prior
    term, and its upstream gradients w.r.t. the rendered maps."""
    lib = _load()
    H, W = cam.height, cam.width
    rgb, depth, sil = _f64(rgb, (3, H, W)), _f64(depth, (H, W)), _f64(sil, (H, W))
    rgb_t, depth_t = _f64(rgb_t, (3, H, W)), _f64(depth_t, (H, W))
    prior = None if prior is None else _f64(prior, (H, W))
    L = ctypes.c_double(0.0)
    d_rgb, d_depth, d_sil = np.zeros((3, H, W)), np.zeros((H, W)), np.zeros((H, W))
    amb = np.zeros((H, W), dtype=np.uint8)
    par = params._c()
    _check(lib.og_loss(ctypes.byref(cam), ctypes.byref(par), _dp(rgb), _dp(depth), _dp(sil), _dp(rgb_t),
                       _dp(depth_t), _dp(prior), ctypes.cast(ctypes.pointer(L), ctypes.POINTER(ctypes.c_double)),
                       _dp(d_rgb), _dp(d_depth), _dp(d_sil), amb.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
           "loss")
    return {"loss": L.value, "d_rgb": d_rgb, "d_depth": d_depth, "d_sil": d_sil, "amb": amb.astype(bool)}


def backward(scene: Scene, cam: Camera, pose, params: Params, d_rgb, d_depth, d_sil) -> dict:
    """Reverse compositing and the chain rule to every parameter and to the pose.

    Returns grads (n x 14: means 3, quats 4, log_scales 3, logit 1, rgb 3), screen
    (n x 10: d mu' 2, d conic 3, d opacity, d rgb 3, d depth) and pose6 = (d theta, d t)
    for the camera turning about its centre (x_c <- Exp(theta) x_c) and shifting
    (x_c <- x_c + t)."""
    lib = _load()
    H, W = cam.height, cam.width
    d_rgb, d_depth, d_sil = _f64(d_rgb, (3, H, W)), _f64(d_depth, (H, W)), _f64(d_sil, (H, W))
    g14 = np.zeros((scene.n, 14))
    g10 = np.zeros((scene.n, 10))
    p6 = np.zeros(6)
    sc, par, pose = scene._c(), params._c(), _f64(pose, (7,))
    _check(lib.og_backward(ctypes.byref(sc), ctypes.byref(cam), _dp(pose), ctypes.byref(par), _dp(d_rgb),
                           _dp(d_depth), _dp(d_sil), _dp(g14), _dp(g10), _dp(p6)), "backward")
    return {"grads": g14, "screen": g10, "pose6": p6}


def adam_step(pose, state, grad6, params: Params):
    """One decoupled rotation / translation Adam step (Sec. III-B); returns (pose, state)."""
    lib = _load()
    pose = _f64(pose, (7,)).copy()
    state = _f64(state, (16,)).copy()
    g = _f64(grad6, (6,))
    par = params._c()
    _check(lib.og_adam_step(_dp(pose), _dp(state), _dp(g), ctypes.byref(par)), "adam_step")
    return pose, state


def num_threads(params: Params) -> int:
    """Threads the oracle's OpenMP loops use with these params."""
    return int(_load().og_num_threads(ctypes.byref(params._c())))
