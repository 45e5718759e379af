"""Helpers for the GPU parity tests: run the CUDA path through the C ABI binding and the
oracle on the same seeded inputs, and compare them the way the tolerances prescribe."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2408_05635_gb300 import gs, scenes

IMG_TOL = 1e-4      # max-abs on colour, depth and silhouette (unambiguous pixels)
GRAD_TOL = 1e-3     # per tensor: ||d||_inf / ||g||_inf and ||d||_2 / ||g||_2


def params_pair(**kw):
    """The same settings for the GPU (gs.Config) and the oracle (oracle.Params)."""
    gcfg = gs.Config(**{k: v for k, v in kw.items() if hasattr(gs.Config, k)})
    op = oracle.Params(**{k: v for k, v in kw.items() if hasattr(oracle.Params, k)})
    return gcfg, op


def ocam(cam):
    return oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)


def gpu_render(R: gs.Rasterizer, gt: gs.GaussianTensors, cams, poses_np, targets=None, margin=1.25):
    poses = torch.tensor(np.asarray(poses_np, dtype=np.float64).reshape(-1, 7), device="cuda")
    prob = R.plan(gt, cams, poses, margin=margin)
    out = R.render(prob, gt, poses, targets=targets)
    counts = R.sync()
    res = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    return res, prob, poses, counts


def split_views(flat, cams, channels):
    """Concatenated planar arrays -> list of per-view (channels, H, W) arrays."""
    out, off = [], 0
    for c in cams:
        n = c.width * c.height * channels
        out.append(flat[off:off + n].reshape(channels, c.height, c.width))
        off += n
    return out


def assert_images_close(gpu, ora, amb, tol=IMG_TOL, what=""):
    ok = ~amb
    diff = np.abs(gpu - ora)
    if diff.ndim == 3:
        diff = diff.max(axis=0)
    worst = diff[ok].max() if ok.any() else 0.0
    assert worst <= tol, f"{what}: max |gpu - oracle| = {worst:.3e} on unambiguous pixels (tol {tol})"


def rel_err(a, b):
    """(inf-norm, 2-norm) of a - b relative to b."""
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    sb = np.abs(b).max()
    if sb == 0:
        return float(np.abs(a).max()), float(np.linalg.norm(a))
    return float(np.abs(a - b).max() / sb), float(np.linalg.norm(a - b) / np.linalg.norm(b))


def assert_grads_close(gpu, ora, tol=GRAD_TOL, what=""):
    ri, r2 = rel_err(gpu, ora)
    assert ri <= tol and r2 <= tol, f"{what}: rel inf {ri:.2e}, rel l2 {r2:.2e} (tol {tol})"
