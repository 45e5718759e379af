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


def check_images(rgb, depth, sil, ref, scene, cam, pose, op, tol=IMG_TOL, what="", max_alt=32) -> dict:
    """GPU maps of one view (planar arrays) against the oracle (ref = oracle.render of the
    same view).  Pixels the oracle does not flag must agree to `tol` in colour, depth and
    silhouette; a flagged pixel must agree to `tol` with one of the outcomes an FP32
    renderer may legitimately produce there (oracle.render_alternatives: the walk of
    Eqs. 2-4 branched at each flagged decision).  Pixels with more outcomes than max_alt
    stay unchecked; their share must stay below 0.01 %.  Returns the shares and errors."""
    H, W = cam.height, cam.width
    rgb, depth, sil = rgb.reshape(3, H, W), depth.reshape(H, W), sil.reshape(H, W)
    err = np.maximum(np.abs(rgb - ref["rgb"]).max(axis=0),
                     np.maximum(np.abs(depth - ref["depth"]), np.abs(sil - ref["sil"])))
    flagged = ref["amb"]
    worst = float(err[~flagged].max()) if (~flagged).any() else 0.0
    assert worst <= tol, f"{what}: max |gpu - oracle| = {worst:.3e} on unflagged pixels (tol {tol})"
    pix = np.flatnonzero(flagged.ravel())
    worst_alt, unresolved = 0.0, 0
    if pix.size:
        alts = oracle.render_alternatives(scene, ocam(cam), pose, op, pix, max_alt=max_alt)
        got = np.stack([rgb[0].ravel()[pix], rgb[1].ravel()[pix], rgb[2].ravel()[pix], depth.ravel()[pix],
                        sil.ravel()[pix]], 1)
        for k, n in enumerate(alts["n_alt"]):
            if n < 1:
                unresolved += 1
                continue
            d = float(np.abs(alts["alts"][k, :n, :5] - got[k]).max(axis=1).min())
            worst_alt = max(worst_alt, d)
            assert d <= tol, f"{what}: flagged pixel {pix[k]} is {d:.3e} from each of its {n} FP32 outcomes"
    share_unres = unresolved / (H * W)
    assert share_unres <= 1e-4, f"{what}: {unresolved} pixels with more than {max_alt} outcomes"
    stats = {"flagged": float(flagged.mean()), "unresolved": share_unres, "max_err_unflagged": worst,
             "max_err_flagged_nearest_outcome": worst_alt}
    print(f"{what}: {stats}")
    return stats


# Relative rounding allowance of the device loss: every pixel's FP32 terms, a 32-lane FP32
# butterfly per warp (5 additions), double-float across warps and tiles: about 9 unit
# roundoffs of 2^-24 relative to the total, taken as 1e-6.
LOSS_ROUNDING = 1e-6


def loss_tolerance(loss, ref, scene, cam, pose, op, rgb_t, depth_t, prior=None, max_alt=32) -> float:
    """Largest |device loss - oracle loss| for an oracle loss `loss`: the FP32 decisions at
    flagged pixels may give another outcome there, so the sum over the flagged pixels of
    the largest change of the pixel's loss term among its FP32 outcomes
    (oracle.render_alternatives; the loss is a sum of per-pixel terms, each evaluated by
    oracle.loss on a one-pixel image), plus LOSS_ROUNDING of the loss.  A pixel with more
    than max_alt outcomes counts with the largest value its term can take (every residual
    at its larger distance to [0, 1] for colour and [0, z_max] for depth, the visibility
    term at its maximum), since both outcomes' terms lie between 0 and that."""
    H, W = cam.height, cam.width
    flagged = ref["amb"].ravel()
    pix = np.flatnonzero(flagged)
    rgb_t = np.asarray(rgb_t, np.float64).reshape(3, H * W)
    depth_t = np.asarray(depth_t, np.float64).reshape(H * W)
    prior = None if prior is None else np.asarray(prior, np.float64).reshape(H * W)
    one = oracle.camera(1.0, 1.0, 0.0, 0.0, 1, 1)

    def term(q, c, d, s):
        return oracle.loss(one, op, np.asarray(c, np.float64).reshape(3, 1, 1), np.full((1, 1), d), np.full((1, 1), s),
                           rgb_t[:, q].reshape(3, 1, 1), depth_t[q:q + 1].reshape(1, 1),
                           None if prior is None else prior[q:q + 1].reshape(1, 1))["loss"]

    total = 0.0
    if pix.size:
        alts = oracle.render_alternatives(scene, ocam(cam), pose, op, pix, max_alt=max_alt)
        rgb_r = ref["rgb"].reshape(3, H * W)
        # no camera-frame depth exceeds |m| + |t| for the scene's means m and the pose's t
        z_max = float(np.linalg.norm(np.asarray(scene.means), axis=1).max() + np.linalg.norm(np.asarray(pose)[4:7]))
        for k, n in enumerate(alts["n_alt"]):
            q = int(pix[k])
            if n < 1:
                pr = 0.0 if prior is None or prior[q] <= 0 else max(prior[q], z_max - prior[q])
                total += (op.w_rgb * np.maximum(rgb_t[:, q], 1.0 - rgb_t[:, q]).sum()
                          + op.w_depth * max(depth_t[q], z_max - depth_t[q]) + op.w_prior * pr + op.w_vis)
                continue
            nom = term(q, rgb_r[:, q], ref["depth"].ravel()[q], ref["sil"].ravel()[q])
            total += max(abs(term(q, a[:3], a[3], a[4]) - nom) for a in alts["alts"][k, :n])
    return total + LOSS_ROUNDING * abs(loss)
