"""Plain FP64 NumPy definitions of the evaluation quantities of Sec. IV on synthetic
sequences: the image sums behind PSNR and the average depth error, and the trajectory
errors (ATE RMSE of the camera centres, rotation angle).

THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU baseline
leg of the benchmark may use it; the product path neither links nor calls it.
"""
from __future__ import annotations

import numpy as np


def image_sums(rgb, depth, rgb_t, depth_t) -> np.ndarray:
    """(sum of squared colour errors, sum |D - D*| over D* > 0, their count, sum (D - D*)^2
    over them)."""
    rgb, rgb_t = np.asarray(rgb, np.float64), np.asarray(rgb_t, np.float64)
    depth, depth_t = np.asarray(depth, np.float64).ravel(), np.asarray(depth_t, np.float64).ravel()
    valid = depth_t > 0
    e = depth[valid] - depth_t[valid]
    return np.array([np.sum((rgb - rgb_t) ** 2), np.sum(np.abs(e)), float(valid.sum()), np.sum(e * e)])


def psnr(sq_sum: float, values: int) -> float:
    """PSNR (dB) of colours in [0, 1] from a sum of squared errors over `values` values."""
    mse = sq_sum / values
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def _rotation(q) -> np.ndarray:
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def camera_centre(pose) -> np.ndarray:
    """World position of the camera of a world->camera pose: c = -R^T t."""
    p = np.asarray(pose, np.float64)
    return -_rotation(p[:4]).T @ p[4:7]


def trajectory_errors(est, gt) -> dict:
    """Per-frame camera-centre distance and rotation angle between estimated and true
    world->camera poses (same world frame, no alignment), and the ATE RMSE."""
    d = np.array([np.linalg.norm(camera_centre(a) - camera_centre(b)) for a, b in zip(est, gt)])
    ang = []
    for a, b in zip(est, gt):
        Rd = _rotation(np.asarray(a)[:4]) @ _rotation(np.asarray(b)[:4]).T
        ang.append(np.arccos(np.clip((np.trace(Rd) - 1.0) / 2.0, -1.0, 1.0)))
    return {"trans": d, "rot": np.array(ang), "ate_rmse": float(np.sqrt(np.mean(d * d)))}
