"""Plain FP64 NumPy oracle of the map-side steps: first-frame initialisation (Sec. III-A),
adding Gaussians where a keyframe shows new observations, the gradient-based update of
every Gaussian parameter with the keyframe poses fixed, and the removal of Gaussians
(Sec. III-C).

THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU baseline
leg of the benchmark may use it; the product path (the CUDA library) neither links nor
calls it and shares no code with it.

Readings where the paper is silent (each a parameter here and a setting on the GPU):
  * a new Gaussian is made for a pixel with a depth measurement (> 0); on a keyframe only
    where the rendered silhouette S is below sil_add (0.5): the silhouette marks what the
    map already explains (Sec. V shows it as the mask of where Gaussians are added);
  * its centre is the pixel's sample point (u, v) unprojected with its depth, its colour
    the pixel's, opacity 0.5 (logit 0), identity rotation and an isotropic scale of
    depth / f with f = (fx + fy) / 2 (a one-pixel radius in the image, Sec. III-A);
  * new Gaussians follow the live ones in row-major pixel order;
  * the parameter update is Adam on the raw parameters with one learning rate per group
    (means, quats, log_scales, logits, rgb), bias-corrected, the optimiser state of a new
    Gaussian starting at zero;
  * duplicate removal drops the Gaussians whose opacity fell below o_min, decided on the
    stored FP32 logit against logit(o_min) rounded to FP32, and keeps the order of the
    others (their optimiser state moves with them).
"""
from __future__ import annotations

import numpy as np

GROUPS = ("means", "quats", "log_scales", "logits", "rgb")
WIDTH = {"means": 3, "quats": 4, "log_scales": 3, "logits": 1, "rgb": 3}


def _rotation(q) -> np.ndarray:
    """World->camera rotation of a unit quaternion (w, x, y, z), renormalised."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def gaussians_from_frame(cam, pose, rgb, depth, sil=None, sil_add: float = 0.5) -> dict:
    """New Gaussians for one RGB-D frame (Sec. III-A; on keyframes, Sec. III-C).

    cam: fx, fy, cx, cy, width, height; pose: 7 values (qw, qx, qy, qz, tx, ty, tz)
    world->camera; rgb 3 x H x W, depth H x W, sil H x W or None (every pixel with depth).
    Returns the parameter groups (n x width each) and `pixel`, the flat index of the pixel
    each Gaussian came from."""
    H, W = int(cam.height), int(cam.width)
    depth = np.asarray(depth, np.float64).reshape(H, W)
    take = depth > 0
    if sil is not None:
        take &= np.asarray(sil, np.float64).reshape(H, W) < sil_add
    pix = np.flatnonzero(take.ravel())
    v, u = np.divmod(pix, W)
    d = depth.ravel()[pix]
    # camera-frame point of the pixel's sample (u, v) at depth d (inverse of pi_m)
    xc = np.stack([(u - cam.cx) / cam.fx * d, (v - cam.cy) / cam.fy * d, d], axis=1)
    R = _rotation(np.asarray(pose, np.float64)[:4])
    t = np.asarray(pose, np.float64)[4:7]
    means = (xc - t) @ R  # R^T (x_c - t), row by row
    f = 0.5 * (cam.fx + cam.fy)
    n = pix.size
    return {"means": means,
            "quats": np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)),
            "log_scales": np.repeat(np.log(d / f)[:, None], 3, axis=1),
            "logits": np.zeros((n, 1)),
            "rgb": np.asarray(rgb, np.float64).reshape(3, H * W)[:, pix].T,
            "pixel": pix}


def adam_step(params: dict, grads: dict, m: dict, v: dict, step: int, lrs: dict, beta1: float, beta2: float,
              eps: float, groups=GROUPS) -> tuple[dict, dict, dict]:
    """One Adam step on every group (Sec. III-C: gradient-based optimisation of the
    Gaussians).  All dicts map a group name to an array; step is the 1-based t; `groups`
    lists the groups present (an isotropic map has no quaternions)."""
    out_p, out_m, out_v = {}, {}, {}
    for k in groups:
        g = np.asarray(grads[k], np.float64)
        mk = beta1 * np.asarray(m[k], np.float64) + (1.0 - beta1) * g
        vk = beta2 * np.asarray(v[k], np.float64) + (1.0 - beta2) * g * g
        m_hat = mk / (1.0 - beta1 ** step)
        v_hat = vk / (1.0 - beta2 ** step)
        out_p[k] = np.asarray(params[k], np.float64) - lrs[k] * m_hat / (np.sqrt(v_hat) + eps)
        out_m[k], out_v[k] = mk, vk
    return out_p, out_m, out_v


def keep_mask(logits, o_min: float) -> np.ndarray:
    """Gaussians that survive duplicate removal: stored FP32 logit >= logit(o_min) in FP32."""
    thr = np.float32(np.log(o_min / (1.0 - o_min)))
    return np.asarray(logits, np.float32).reshape(-1) >= thr


def prune(arrays: dict, logits, o_min: float) -> dict:
    """Stable compaction of every array (rows = Gaussians) to the kept Gaussians."""
    keep = keep_mask(logits, o_min)
    return {k: np.asarray(a)[keep] for k, a in arrays.items()}
