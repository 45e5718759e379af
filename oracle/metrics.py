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


# ---------------------------------------------------------------------------- MS-SSIM

# Multi-scale structural similarity (Wang, Simoncelli and Bovik, 2003): per scale the
# contrast-structure term cs = (2 s_xy + C2) / (s_x^2 + s_y^2 + C2) averaged over the
# image, on the coarsest scale also the luminance term l = (2 m_x m_y + C1) /
# (m_x^2 + m_y^2 + C1); local statistics under an 11 x 11 Gaussian window (sigma 1.5) over
# the window positions that fit (valid); 2 x 2 average pooling between the five scales;
# MS-SSIM = l_5^b5 prod_j cs_j^bj with the published exponents.  Readings: colours in
# [0, 1] (L = 1), K1 = 0.01, K2 = 0.03; negative cs clamped at 0; computed per colour
# channel and averaged over the channels.
MSSSIM_WEIGHTS = (0.0448, 0.2856, 0.3001, 0.2363, 0.1333)


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _filter_valid(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Separable correlation with the window, valid positions only."""
    k = g.size
    H, W = img.shape
    rows = np.zeros((H, W - k + 1))
    for j in range(k):
        rows += g[j] * img[:, j:j + W - k + 1]
    out = np.zeros((H - k + 1, W - k + 1))
    for i in range(k):
        out += g[i] * rows[i:i + H - k + 1, :]
    return out


def ssim_terms(x: np.ndarray, y: np.ndarray, k1: float = 0.01, k2: float = 0.03) -> tuple[float, float]:
    """(mean l, mean cs) of two single-channel images at one scale."""
    g = gaussian_window()
    c1, c2 = k1 * k1, k2 * k2
    mx, my = _filter_valid(x, g), _filter_valid(y, g)
    sxx = _filter_valid(x * x, g) - mx * mx
    syy = _filter_valid(y * y, g) - my * my
    sxy = _filter_valid(x * y, g) - mx * my
    l = (2 * mx * my + c1) / (mx * mx + my * my + c1)
    cs = (2 * sxy + c2) / (sxx + syy + c2)
    return float(l.mean()), float(cs.mean())


def _pool2(img: np.ndarray) -> np.ndarray:
    H, W = img.shape[0] // 2, img.shape[1] // 2
    return 0.25 * (img[0:2 * H:2, 0:2 * W:2] + img[1:2 * H:2, 0:2 * W:2] + img[0:2 * H:2, 1:2 * W:2]
                   + img[1:2 * H:2, 1:2 * W:2])


def ms_ssim(rgb, rgb_t) -> dict:
    """MS-SSIM of two colour images (3 x H x W in [0, 1]): per channel and the mean."""
    rgb, rgb_t = np.asarray(rgb, np.float64), np.asarray(rgb_t, np.float64)
    per = []
    for ch in range(rgb.shape[0]):
        x, y = rgb[ch], rgb_t[ch]
        val = 1.0
        for j, b in enumerate(MSSSIM_WEIGHTS):
            l, cs = ssim_terms(x, y)
            val *= max(cs, 0.0) ** b
            if j == len(MSSSIM_WEIGHTS) - 1:
                val *= max(l, 0.0) ** b
            else:
                x, y = _pool2(x), _pool2(y)
        per.append(val)
    return {"ms_ssim": float(np.mean(per)), "per_channel": per}
