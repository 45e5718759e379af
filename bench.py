"""Benchmark: fwd+bwd render Mpix/s and tracking iterations/s of the differentiable
3D-Gaussian rasterizer on the 640 x 480, 200k-Gaussian room (plain FP32 attributes).

One step = one full tracking iteration of the hot path on one frame (every 40 steps the
pose restarts from the frame's start pose, as tracking a new frame would): projection and
tile binning, per-tile depth sort, front-to-back compositing of colour / depth /
silhouette with the fused combined loss, reverse compositing, chain rule to the pose,
FP64 pose reduction and the decoupled Adam update (all CUDA kernels of this library,
launched from the library's CUDA graph).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Rank 0 prints one JSON line.  With N > 1 (torchrun) every rank tracks its own frame:
replicas only, weak scaling.  ``--impl reference`` times the FP64 CPU oracle on the
same workload (bounded samples per step) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd render Mpix/s & tracking iters/s (640×480, 200k Gauss) vs plain"
WORKLOAD = "tracking 640x480, 200k room Gaussians, fp32 attributes"
N_GAUSS = 200_000
# FP32 operations (an FMA counts 2, an ex2 or reciprocal 1) of one differentiated
# (pixel, Gaussian) pair in the pose-gradient backward and of one contributing pair in
# the forward: the per-unit algorithmic work of the two compositing kernels.
FLOP_BWD_PAIR = 58
FLOP_FWD_PAIR = 23
FLOP_BPROJ_REC = 300  # about: the chain rule of one record to the pose (k_bproject, pose only)
FP32_LANES = 128  # FP32 FMA lanes per SM (Blackwell)
ITERS_PER_FRAME = 40  # tracking iterations per frame (the 640 x 480 tracking workload); the
                      # pose and Adam state restart from the frame's start pose every 40 steps


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--batched-steps", type=int, default=10,
                    help="timed steps of the batched BF16 hypothesis leg (0 skips it)")
    ap.add_argument("--mapping-steps", type=int, default=5,
                    help="timed windows of the mapping leg (0 skips it)")
    ap.add_argument("--sequence-frames", type=int, default=200,
                    help="frames of the long-sequence leg (0 skips it)")
    ap.add_argument("--isotropic-steps", type=int, default=400,
                    help="timed steps of the isotropic-versus-anisotropic leg (0 skips it)")
    ap.add_argument("--autotune-reps", type=int, default=10,
                    help="passes per setting of the launch-schedule autotuner before the tracking and batched "
                         "legs (0: the default schedule)")
    ap.add_argument("--schedule", default=None,
                    help="fixed launch schedule 'tile_w,tile_h,sub_buckets,fwd_batch,bwd_batch[,flags]' instead of "
                         "tuning (flags 1: the fused tracking compositor)")
    return ap.parse_args()


def apply_schedule(a, R, cams, g, poses, targets) -> dict:
    """The launch schedule of a leg: fixed by --schedule, else picked by the library's
    autotuner on the leg's own views (gs_autotune), else the default.  The tuning problem
    gets twice the usual pair-capacity margin, so that smaller tiles, which make more
    (Gaussian, tile) pairs, are timed too; the leg plans its own problem afterwards."""
    if a.schedule:
        R.set_schedule(*(int(x) for x in a.schedule.split(",")))
        return {"schedule": R.schedule, "tuned": False}
    if a.autotune_reps > 0:
        tprob = R.plan(g, cams, poses, margin=3.0)
        res = R.autotune(tprob, g, poses, targets, pose_only=True, reps=a.autotune_reps)
        res["tuned"] = True
        return res
    return {"schedule": R.schedule, "tuned": False}


def workload(seed: int = 0):
    """Synthetic stand-in for a TUM RGB-D tracking frame (the dataset is not available):
    the room scene, the ground-truth camera, a start pose 2 deg / 5 cm away, an RGB-D
    frame ray-cast from the ground truth and a depth prior (x (1 + N(0, 0.02)), 5% holes)."""
    from paper_2408_05635_gb300 import scenes
    g = scenes.room_scene(N_GAUSS, seed=seed)
    cam = scenes.TUM_CAM
    gt = scenes.tracking_gt_pose()
    rng = np.random.default_rng(seed + 1)
    start = scenes.perturb_pose(gt, rng, 2.0, 0.05)
    rgb, depth = scenes.raycast_room(gt, cam, seed=seed)
    prior = scenes.prior_from_depth(depth, rng, 0.02, 0.05)
    return g, cam, gt, start, rgb, depth, prior


N_BATCH_GAUSS = 500_000
BATCH_FRAMES, BATCH_HYP = 32, 16


def batched_workload(seed: int = 0):
    """Pose hypotheses over keyframes of uneven resolution: 32 keyframes (320 x 240, 640 x 480
    or 1200 x 680), 16 hypotheses each (rotation N(0, 2 deg), translation N(0, 4 cm)), a
    500k-Gaussian room; each keyframe's RGB-D target is ray-cast from its ground truth, with
    a depth prior (x (1 + N(0, 0.02)), 5% holes)."""
    from paper_2408_05635_gb300 import scenes
    g = scenes.room_scene(N_BATCH_GAUSS, seed=seed)
    cams, poses, frame_of, gts, frame_cams = scenes.batched_keyframes(BATCH_FRAMES, BATCH_HYP, seed=seed)
    rng = np.random.default_rng(seed + 2)
    frames = []
    for f in range(BATCH_FRAMES):
        rgb, depth = scenes.raycast_room(gts[f], frame_cams[f], seed=seed)
        frames.append((rgb, depth, scenes.prior_from_depth(depth, rng, 0.02, 0.05)))
    return g, cams, poses, frame_of, frames


N_MAP_GAUSS = 1_000_000
MAP_VIEWS = 8


def mapping_workload(seed: int = 0):
    """A mapping window (Sec. III-C: keyframe poses fixed, Gaussians optimised): 8 keyframes
    of 1200 x 680 on a circle around the room centre, 45 deg of yaw apart, over a 1M-Gaussian
    room; RGB-D targets ray-cast from the keyframe poses, depth priors (x (1 + N(0, 0.03)),
    8% holes)."""
    from paper_2408_05635_gb300 import scenes
    g = scenes.room_scene(N_MAP_GAUSS, seed=seed)
    poses = np.asarray(scenes.mapping_keyframes(MAP_VIEWS))
    cams = [scenes.WIDE_CAM] * MAP_VIEWS
    rng = np.random.default_rng(seed + 3)
    frames = []
    for v in range(MAP_VIEWS):
        rgb, depth = scenes.raycast_room(poses[v], cams[v], seed=seed)
        frames.append((rgb, depth, scenes.prior_from_depth(depth, rng, 0.03, 0.08)))
    return g, cams, poses, frames


def run_mapping(a, dev, stream):
    """Map-gradient windows: the combined loss of every keyframe of the window rendered and
    differentiated to all 14 parameters of every Gaussian, `chunk` views per call through
    one workspace (a larger chunk fills the GPU better, a smaller one needs less memory)."""
    import torch
    from paper_2408_05635_gb300 import gs
    g, cams, poses_np, frames = mapping_workload()
    poses = torch.tensor(poses_np, dtype=torch.float64, device=dev)
    targets = [tuple(torch.from_numpy(x).to(dev) for x in f) for f in frames]
    gt = gs.GaussianTensors.from_numpy(g, device=dev)
    P = sum(c.width * c.height for c in cams)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    res, loss_v = {}, None
    for chunk in (1, 2, 4, 8):
        R = gs.Rasterizer(gs.Config(), device=dev)
        probs = [R.plan(gt, cams[v0:v0 + chunk], poses[v0:v0 + chunk].contiguous(), margin=1.25)
                 for v0 in range(0, MAP_VIEWS, chunk)]
        ws_bytes = max(gs.gs_workspace_size(R.ctx, pr) for pr in probs)
        grads = None
        with torch.cuda.stream(stream):
            for _ in range(2):
                out = R.mapping_grads(gt, cams, poses, targets, chunk=chunk, probs=probs, stream=stream)
                grads = out["grads"]
            torch.cuda.synchronize(dev)
            ev[0].record(stream)
            for _ in range(a.mapping_steps):
                for t in grads.values():
                    t.zero_()
                out = R.mapping_grads(gt, cams, poses, targets, chunk=chunk, grads=grads, probs=probs, stream=stream)
            ev[1].record(stream)
        torch.cuda.synchronize(dev)
        R.sync(stream)
        ms = ev[0].elapsed_time(ev[1]) / a.mapping_steps
        res[chunk] = {"ms_per_window": round(ms, 3), "mpix_per_s": round(P / ms / 1e3, 1),
                      "workspace_gb": round(ws_bytes / 1e9, 2)}
        loss_v = out["loss"].cpu().numpy()
        R.close()
    best = min(res, key=lambda c: res[c]["ms_per_window"])
    return {"workload": f"{MAP_VIEWS} keyframes 1200x680, {N_MAP_GAUSS // 1000}k room Gaussians, fp32, "
                        "gradients of all 14 parameters",
            "pixels_per_window": P, "chunks": {str(c): v for c, v in res.items()}, "best_chunk": best,
            "loss_per_view": [round(float(x), 5) for x in loss_v],
            "l2": "working set far above L2 (no flush)"}


N_SEQ_GAUSS = 2_000_000


def sequence_workload(dev, n_frames: int, seed: int = 0):
    """The long sequence: 640 x 480 frames along a closed spline around the room (1.8 deg
    and 4 cm per frame on average), each an RGB-D frame ray-cast from the true pose (on the
    GPU) with a depth prior (x (1 + N(0, 0.02)), 5% holes); the 2M-Gaussian room as the
    fixed map for the tracking-only run, with FP16 attributes."""
    import torch
    from paper_2408_05635_gb300 import scenes
    g = scenes.room_scene(N_SEQ_GAUSS, seed=seed)
    cam = scenes.TUM_CAM
    poses = scenes.spline_trajectory(n_frames, seed=seed)
    gen = torch.Generator(device=dev).manual_seed(seed + 5)
    frames = []
    for p in poses:
        rgb, depth = scenes.raycast_room_torch(p, cam, seed=seed, device=dev)
        noise = torch.randn(depth.shape, generator=gen, device=dev) * 0.02
        holes = torch.rand(depth.shape, generator=gen, device=dev) < 0.05
        prior = torch.where(holes, torch.zeros_like(depth), depth * (1 + noise))
        frames.append((rgb, depth, prior))
    return g, cam, poses, frames


def _trajectory_report(est, gt):
    from paper_2408_05635_gb300 import scenes, slam
    ce, cg = slam.camera_centres(est), slam.camera_centres(gt)
    d = np.linalg.norm(ce - cg, axis=1)
    ang = []
    for a, b in zip(est, gt):
        Ra, Rb = scenes.pose_rt(a)[0], scenes.pose_rt(b)[0]
        ang.append(np.degrees(np.arccos(np.clip((np.trace(Ra @ Rb.T) - 1) / 2, -1, 1))))
    return {"ate_rmse_cm": round(100 * float(np.sqrt(np.mean(d * d))), 3), "max_trans_err_cm": round(100 * float(d.max()), 3),
            "final_trans_err_cm": round(100 * float(d[-1]), 3), "max_rot_err_deg": round(float(np.max(ang)), 4)}


def run_sequence(a, dev, stream):
    """Tracking over a long sequence: on the fixed true map (every frame started from the
    previous estimate, 100 iterations in one graph launch), and the whole loop from an
    empty map (first-frame Gaussians, tracking, keyframe additions, window optimisation
    and removal)."""
    import time
    import torch
    from paper_2408_05635_gb300 import gs, slam
    g, cam, gt_poses, frames = sequence_workload(dev, a.sequence_frames)
    F = len(gt_poses)
    P = cam.width * cam.height
    out = {"workload": f"{F} frames 640x480 along a spline around the room, 100 tracking iterations per frame"}
    # (1) tracking on the fixed 2M-Gaussian map, FP16 attributes
    gt = gs.GaussianTensors.from_numpy(g, device=dev, attr_dtype=torch.float16)
    tr = slam.Tracker(cam, 100, device=dev, autotune_reps=a.autotune_reps)
    pose = torch.tensor(gt_poses[0], dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        tr.track(gt, pose, *frames[1], stream=stream)  # plan and capture
        torch.cuda.synchronize(dev)
        est = [pose.clone()]
        t0 = time.perf_counter()
        for k in range(1, F):
            pose = tr.track(gt, est[-1], *frames[k], stream=stream)
            est.append(pose)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    tr.close()
    rep = _trajectory_report(torch.stack(est).cpu().numpy(), gt_poses)
    out["tracking_fixed_map"] = {"map": f"{N_SEQ_GAUSS // 1000}k room Gaussians, fp16 attributes",
                                 "ms_per_frame": round(1e3 * wall / (F - 1), 3),
                                 "tracking_iters_per_s": round(100 * (F - 1) / wall, 1),
                                 "mpix_per_s": round(100 * (F - 1) * P / wall / 1e6, 1), "replans": tr.replans,
                                 "launch_schedule": tr.tune["schedule"] if tr.tune else tr.R.schedule, **rep}
    del gt
    # (2) the whole loop from an empty map, with anisotropic Gaussians and with the
    # isotropic ones of Eq. 1 as written
    for key, iso in (("slam_from_empty_map", False), ("slam_from_empty_map_isotropic", True)):
        cfg = slam.SlamConfig(lowp=torch.float16, isotropic=iso, autotune_reps=a.autotune_reps)
        S = slam.Slam(cam, cfg, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(F):
                S.process(k, *frames[k], first_pose=gt_poses[0] if k == 0 else None, stream=stream)
            torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        rep = _trajectory_report(torch.stack(S.poses).cpu().numpy(), gt_poses)
        q = S.evaluate(frames, stream)
        out[key] = {"ms_per_frame": round(1e3 * wall / F, 3), "frames_per_s": round(F / wall, 2),
                    "keyframes": S.stats["keyframes"], "map_iters_per_keyframe": cfg.map_iters,
                    "first_frame_map_iters": cfg.first_map_iters, "window": cfg.window, "final_map_gaussians": S.n,
                    "added_total": int(sum(S.stats["added"])), "pruned_total": int(sum(S.stats["pruned"])),
                    "replans": S.tracker.replans, "schedule_tunings": S.tracker.tunes,
                    "launch_schedule": S.tracker.R.schedule, **rep, **{k: round(v, 3) for k, v in q.items()}}
        S.close()
        del S
    return out


def run_isotropic(dev, stream, steps: int = 400):
    """The same tracking iteration with the room stored as isotropic Gaussians (Eq. 1 as
    written: 32 bytes per Gaussian instead of 56; radius = geometric mean of the scales),
    beside the anisotropic store, each warm and with the L2 flushed between steps."""
    import torch
    from paper_2408_05635_gb300 import gs, scenes
    g, cam, gt_pose, start, rgb, depth, prior = workload()
    iso = scenes.Gaussians(g.means, None, g.log_scales.mean(axis=1, keepdims=True).astype(np.float32), g.logits, g.rgb)
    tg_t = [torch.tensor(x.reshape(-1), device=dev) for x in (rgb, depth, prior)]
    tg = gs.gs_targets(*(x.data_ptr() for x in tg_t))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for name, gg in (("anisotropic", g), ("isotropic", iso)):
        R = gs.Rasterizer(gs.Config(), device=dev)
        gt = gs.GaussianTensors.from_numpy(gg, device=dev)
        poses = torch.tensor(np.asarray(start)[None], dtype=torch.float64, device=dev)
        prob = R.plan(gt, [cam], poses, margin=1.5)
        ws, nb = R.workspace(prob)
        adam = torch.zeros(1, 16, dtype=torch.float64, device=dev)
        loss = torch.zeros(1, 1, dtype=torch.float64, device=dev)
        s0 = poses.clone()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
        for k in range(steps + 5):
            if k % ITERS_PER_FRAME == 0:
                poses.copy_(s0)
                adam.zero_()
            flush.fill_(float(k))
            j = k - 5
            if j >= 0:
                ev[2 * j].record(stream)
            gs.gs_track_step(R.ctx, prob, gt.c(), tg, poses, adam, loss, 1, ws, nb, stream)
            if j >= 0:
                ev[2 * j + 1].record(stream)
        torch.cuda.synchronize(dev)
        R.sync(stream)
        us = 1e3 * sum(ev[2 * j].elapsed_time(ev[2 * j + 1]) for j in range(steps)) / steps
        res[name] = {"us_per_iter": round(us, 2), "bytes_per_gaussian": 32 if name == "isotropic" else 56}
        R.close()
    res["workload"] = "tracking 640x480, the 200k room (isotropic: radius = geometric mean of the scales)"
    return res


def run_batched(a, dev, stream, mhz: float = 2070.0):
    """The batched / low-precision form beside the plain one, on the same views, with the
    two changes separated: all 512 hypotheses tracked in one call with BF16 attributes and
    with FP32 attributes (each with its launch schedule tuned on the 512-view problem), and
    the same keyframes' views tracked one call per view with FP32 attributes (one
    hypothesis per keyframe), on the default schedule and tuned per resolution."""
    import torch
    from paper_2408_05635_gb300 import gs
    g, cams, poses0, frame_of, frames = batched_workload()
    V = len(cams)
    pix = [c.width * c.height for c in cams]
    P = sum(pix)
    # targets of every view, in view order (a keyframe's target repeated for its hypotheses)
    t_rgb = torch.cat([torch.from_numpy(frames[f][0].reshape(-1)) for f in frame_of]).to(dev)
    t_depth = torch.cat([torch.from_numpy(frames[f][1].reshape(-1)) for f in frame_of]).to(dev)
    t_prior = torch.cat([torch.from_numpy(frames[f][2].reshape(-1)) for f in frame_of]).to(dev)
    start = torch.tensor(np.asarray(poses0), dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def track(R, gt, prob, ws, nb, poses, adam, loss, targets):
        gs.gs_track_step(R.ctx, prob, gt.c(), targets, poses, adam, loss, 1, ws, nb, stream)

    def batched(attr_dtype):
        """One call over all views; returns the timings and the pose gradients at the start."""
        R = gs.Rasterizer(gs.Config(), device=dev)
        gtb = gs.GaussianTensors.from_numpy(g, device=dev, attr_dtype=attr_dtype)
        poses = start.clone()
        sched = apply_schedule(a, R, cams, gtb, poses, (t_rgb, t_depth, t_prior))
        prob = R.plan(gtb, cams, poses, margin=1.5)
        ws, nb = R.workspace(prob)
        tg = gs.gs_targets(t_rgb.data_ptr(), t_depth.data_ptr(), t_prior.data_ptr())
        adam = torch.zeros(V, 16, dtype=torch.float64, device=dev)
        loss = torch.zeros(1, V, dtype=torch.float64, device=dev)
        for _ in range(3):
            track(R, gtb, prob, ws, nb, poses, adam, loss, tg)
        gs.gs_set_profiling(R.ctx, True)
        track(R, gtb, prob, ws, nb, poses, adam, loss, tg)
        kms = dict(gs.gs_kernel_times(R.ctx))
        gs.gs_set_profiling(R.ctx, False)
        _, cb = gs.gs_sync_status(R.ctx, stream)  # the work of that iteration, counted on the device
        bytes_attr = 22 if attr_dtype == torch.bfloat16 else 44
        rl = kernel_rooflines(kms, N_BATCH_GAUSS, V, bytes_attr, int(cb.n_records), int(cb.n_pairs),
                              int(cb.fwd_contrib), int(cb.bwd_contrib), mhz)
        poses.copy_(start)
        adam.zero_()
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for _ in range(a.batched_steps):
            track(R, gtb, prob, ws, nb, poses, adam, loss, tg)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        st, _ = gs.gs_sync_status(R.ctx, stream)
        if st:
            raise SystemExit(f"batched leg: device reported {gs._STATUS[st]}")
        ms = ev[0].elapsed_time(ev[1]) / a.batched_steps
        poses.copy_(start)
        R.render(prob, gtb, poses, targets=(t_rgb, t_depth, t_prior), stream=stream, images=False)
        grad = R.backward(gtb, params=False, pose=True, stream=stream, n_views=V)["pose_grad"].clone()
        res = {"ms_per_step": ms, "view_iters_per_s": V / (ms / 1e3), "mpix_per_s": P / ms / 1e3,
               "launch": "one gs_track_step call (one CUDA graph) for all views",
               "kernels_us": {k: round(1e3 * v, 1) for k, v in kms.items()}, "roofline_kernels": rl,
               "launch_schedule": sched, "pairs": int(cb.n_pairs), "workspace_gb": round(nb / 1e9, 2)}
        R.close()
        del ws
        return res, grad

    b16, g_b16 = batched(torch.bfloat16)
    b32, g_b32 = batched(torch.float32)

    # plain: one hypothesis per keyframe, one call per view, FP32 attributes
    gtf = gs.GaussianTensors.from_numpy(g, device=dev, attr_dtype=torch.float32)
    sub = [int(np.flatnonzero(frame_of == f)[0]) for f in range(BATCH_FRAMES)]
    off = np.concatenate([[0], np.cumsum(pix)])
    sub_pix = sum(pix[v] for v in sub)

    def plain(tuned):
        Rs, scheds = {}, {}
        total_ms, grads = 0.0, {}
        reps = 10
        for v in sub:
            res_key = (cams[v].width, cams[v].height)
            tr = (t_rgb[3 * off[v]:3 * off[v + 1]], t_depth[off[v]:off[v + 1]], t_prior[off[v]:off[v + 1]])
            if res_key not in Rs:  # one context per resolution, tuned on its first view
                Rs[res_key] = gs.Rasterizer(gs.Config(), device=dev)
                if tuned and a.autotune_reps > 0:
                    pv = start[v:v + 1].clone()
                    tp = Rs[res_key].plan(gtf, [cams[v]], pv, margin=3.0)
                    Rs[res_key].autotune(tp, gtf, pv, tr, pose_only=True, reps=a.autotune_reps)
                scheds[f"{res_key[0]}x{res_key[1]}"] = Rs[res_key].schedule
            Rp = Rs[res_key]
            pv = start[v:v + 1].clone()
            pr = Rp.plan(gtf, [cams[v]], pv, margin=1.5)
            wsv, nbv = Rp.workspace(pr)
            tgv = gs.gs_targets(tr[0].data_ptr(), tr[1].data_ptr(), tr[2].data_ptr())
            av = torch.zeros(1, 16, dtype=torch.float64, device=dev)
            lv = torch.zeros(1, 1, dtype=torch.float64, device=dev)
            track(Rp, gtf, pr, wsv, nbv, pv, av, lv, tgv)  # captures this view's graph
            torch.cuda.synchronize(dev)
            ev[0].record(stream)
            for _ in range(reps):
                track(Rp, gtf, pr, wsv, nbv, pv, av, lv, tgv)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            total_ms += ev[0].elapsed_time(ev[1]) / reps
            pv.copy_(start[v:v + 1])
            Rp.render(pr, gtf, pv, targets=tr, stream=stream, images=False)
            grads[v] = Rp.backward(gtf, params=False, pose=True, stream=stream)["pose_grad"][0].clone()
        for Rp in Rs.values():
            Rp.close()
        return {"views_timed": len(sub), "ms_per_view_iter": total_ms / len(sub),
                "view_iters_per_s": len(sub) / (total_ms / 1e3), "mpix_per_s": sub_pix / total_ms / 1e3,
                "launch": "one gs_track_step call per view", "launch_schedule": scheds}, grads

    p_def, g_f = plain(False)
    p_tuned, _ = plain(True)

    def rel(gb):
        r = [float((gb[v] - g_f[v]).norm() / g_f[v].norm().clamp_min(1e-30)) for v in sub]
        return {"max": max(r), "median": float(np.median(r))}

    return {
        "workload": f"{BATCH_FRAMES} keyframes x {BATCH_HYP} pose hypotheses (uneven 320x240 / 640x480 / "
                    f"1200x680), {N_BATCH_GAUSS // 1000}k room Gaussians",
        "views": V, "pixels_per_step": P,
        "batched_bf16": b16, "batched_fp32": b32,
        "plain_fp32": p_def, "plain_fp32_tuned": p_tuned,
        "speedup_batching": b32["view_iters_per_s"] / p_tuned["view_iters_per_s"],
        "speedup_bf16_attributes": b16["view_iters_per_s"] / b32["view_iters_per_s"],
        "speedup_view_iters": b16["view_iters_per_s"] / p_def["view_iters_per_s"],
        "speedup_vs_tuned_plain": b16["view_iters_per_s"] / p_tuned["view_iters_per_s"],
        "pose_grad_rel_diff_bf16_vs_fp32": rel(g_b16),
        "pose_grad_rel_diff_batched_fp32_vs_plain_fp32": rel(g_b32),
        "l2": "working set far above L2 (no flush)",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:  # first sample before timing starts
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(g, cam, start, rgb, depth, prior, budget_s: float):
    """The FP64 oracle's tracking iteration (render, loss, backward, Adam step) on the
    host cores, repeated on the same frame until `budget_s` seconds have elapsed."""
    import oracle
    p = oracle.Params()
    sc = oracle.Scene(*g.arrays())
    oc = oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    pose, state = np.asarray(start, np.float64).copy(), np.zeros(16)
    iters, t0 = 0, time.perf_counter()
    while True:
        r = oracle.render(sc, oc, pose, p)
        L = oracle.loss(oc, p, r["rgb"], r["depth"], r["sil"], rgb, depth, prior)
        b = oracle.backward(sc, oc, pose, p, L["d_rgb"], L["d_depth"], L["d_sil"])
        pose, state = oracle.adam_step(pose, state, b["pose6"], p)
        iters += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    its = iters / el
    return {"value": its * cam.width * cam.height / 1e6, "unit": "Mpix/s", "iters_per_s": its,
            "cores": oracle.num_threads(p), "kind": "oracle",
            "sample": f"{iters} full tracking iterations of the 640x480 / 200k workload in {el:.1f} s"}


def _check_view(sc, oc, pose, op, ref, rgb, depth, sil, max_alt=32):
    """A GPU view (planar maps) against the oracle's: the largest error on pixels the oracle
    does not flag, and on flagged pixels the distance to the nearest of the outcomes an
    FP32 renderer may legitimately produce there (the walk of Eqs. 2-4 branched at each
    flagged decision); pixels with more than max_alt outcomes are counted as unchecked."""
    import oracle
    H, W = oc.height, oc.width
    rgb, depth, sil = rgb.reshape(3, H, W), depth.reshape(H, W), sil.reshape(H, W)
    err = np.maximum(np.abs(rgb - ref["rgb"]).max(axis=0),
                     np.maximum(np.abs(depth - ref["depth"]), np.abs(sil - ref["sil"])))
    flagged = ref["amb"]
    pix = np.flatnonzero(flagged.ravel())
    near, unres = 0.0, 0
    if pix.size:
        A = oracle.render_alternatives(sc, oc, pose, op, pix, max_alt=max_alt)
        got = np.stack([rgb[0].ravel()[pix], rgb[1].ravel()[pix], rgb[2].ravel()[pix], depth.ravel()[pix],
                        sil.ravel()[pix]], 1)
        for k, n in enumerate(A["n_alt"]):
            if n < 1:
                unres += 1
            else:
                near = max(near, float(np.abs(A["alts"][k, :n, :5] - got[k]).max(axis=1).min()))
    return {"max_err_unflagged": float(err[~flagged].max()) if (~flagged).any() else 0.0,
            "flagged_share": float(flagged.mean()), "max_err_flagged_nearest_outcome": near,
            "unchecked_share": unres / (H * W)}


def _rel(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return {"inf": float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)),
            "l2": float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))}


def _masked_upstream(ref, L):
    m = ref["amb"] | L["amb"]
    return [np.where(m[None], 0.0, L["d_rgb"]), np.where(m, 0.0, L["d_depth"]), np.where(m, 0.0, L["d_sil"])], m


def _view_accuracy(dev, stream, g_np, g_oracle, cam, pose, targets, attr_dtype, params_grads=False):
    """One view rendered and differentiated by the GPU (attributes in attr_dtype) and by
    the oracle on g_oracle (the attributes the GPU reads): images, loss, and the pose
    gradient (and with params_grads every parameter gradient) for the oracle's loss
    gradient with flagged pixels zeroed as the shared upstream; and the pose gradient
    through each side's own fused loss."""
    import torch
    import oracle
    from paper_2408_05635_gb300 import gs
    op = oracle.Params()
    sc = oracle.Scene(*g_oracle.arrays())
    oc = oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    rgb_t, depth_t, prior_t = targets
    ref = oracle.render(sc, oc, pose, op)
    L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], rgb_t, depth_t, prior_t)
    ups, mask = _masked_upstream(ref, L)
    ob = oracle.backward(sc, oc, pose, op, *ups)
    of = oracle.backward(sc, oc, pose, op, L["d_rgb"], L["d_depth"], L["d_sil"])
    R = gs.Rasterizer(gs.Config(), device=dev)
    gt = gs.GaussianTensors.from_numpy(g_np, device=dev, attr_dtype=attr_dtype)
    poses = torch.tensor(np.asarray(pose)[None], dtype=torch.float64, device=dev)
    tt = tuple(torch.tensor(np.ascontiguousarray(x).reshape(-1), dtype=torch.float32, device=dev)
               for x in (rgb_t, depth_t, prior_t))
    prob = R.plan(gt, [cam], poses, margin=1.5)
    out = R.render(prob, gt, poses, targets=tt, stream=stream)
    fused = R.backward(gt, params=False, pose=True, stream=stream)["pose_grad"][0].cpu().numpy()
    R.render(prob, gt, poses, stream=stream, images=False)
    upt = tuple(torch.tensor(u.reshape(-1).astype(np.float32), device=dev) for u in ups)
    b = R.backward(gt, upstream=upt, params=params_grads, pose=True, stream=stream)
    parts = gs.gs_pose_partials(R.ctx, stream)
    R.sync(stream)
    res = _check_view(sc, oc, pose, op, ref, *(out[k].cpu().numpy().astype(np.float64) for k in ("rgb", "depth", "sil")))
    res["loss_rel_err"] = abs(float(out["loss"][0]) - L["loss"]) / abs(L["loss"])
    pg = b["pose_grad"][0].cpu().numpy()
    res["pose_grad_rel_err"] = _rel(pg, ob["pose6"])
    res["pose_grad_fused_loss_rel_err"] = _rel(fused, of["pose6"])
    res["masked_upstream_share"] = float(mask.mean())
    # the double-float pose reduction against an FP64 sum of the same per-cell partials
    import math
    exact = [math.fsum(float(h) + float(lo) for h, lo in parts[:, k, :]) for k in range(6)]
    res["pose_reduction_df_vs_fp64_rel"] = _rel(pg, exact)["inf"]
    if params_grads:
        names = [("means", 0, 3), ("quats", 3, 7), ("log_scales", 7, 10), ("logits", 10, 11), ("rgb", 11, 14)]
        res["param_grad_rel_err"] = {n: _rel(b["grads"][n].cpu().numpy().reshape(g_np.n, -1), ob["grads"][:, lo:hi])
                                     for n, lo, hi in names}
    R.close()
    return res, fused


def sequence_drift(dev, stream, frames_n: int = 10, iters: int = 100):
    """Pose drift of the GPU tracker against the oracle's own tracking loop: the first
    `frames_n` frames of the long sequence's 200-frame spline path at 160 x 120, a 200k-Gaussian room
    with FP16 attributes (the oracle on their FP32 values), `iters` decoupled Adam
    iterations per frame, each frame started from that side's previous estimate."""
    import torch
    import oracle
    from paper_2408_05635_gb300 import gs, scenes, slam
    g = scenes.room_scene(200_000, seed=3)
    cam = scenes.Cam(131.25, 131.25, 79.5, 59.5, 160, 120)
    poses = scenes.spline_trajectory(200, seed=0)[:frames_n + 1]  # the 200-frame path's first frames
    gq = scenes.Gaussians(g.means, *(torch.tensor(a).to(torch.float16).float().numpy() for a in
                                     (g.quats, g.log_scales, g.logits, g.rgb)))
    rng = np.random.default_rng(11)
    frames = []
    for p in poses:
        rgb, depth = scenes.raycast_room(p, cam, seed=3)
        frames.append((rgb, depth, scenes.prior_from_depth(depth, rng, 0.02, 0.05)))
    gt = gs.GaussianTensors.from_numpy(g, device=dev, attr_dtype=torch.float16)
    tr = slam.Tracker(cam, iters, device=dev)
    est_gpu = [np.asarray(poses[0], np.float64)]
    with torch.cuda.stream(stream):
        for k in range(1, frames_n + 1):
            f = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in frames[k]]
            start = torch.tensor(est_gpu[-1], dtype=torch.float64, device=dev)
            est_gpu.append(tr.track(gt, start, *f, stream=stream).cpu().numpy().reshape(7))
    tr.close()
    op = oracle.Params()
    sc = oracle.Scene(*gq.arrays())
    oc = oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    est_o = [np.asarray(poses[0], np.float64)]
    t0 = time.perf_counter()
    for k in range(1, frames_n + 1):
        pose, state = est_o[-1].copy(), np.zeros(16)
        rgb, depth, prior = frames[k]
        for _ in range(iters):
            r = oracle.render(sc, oc, pose, op)
            L = oracle.loss(oc, op, r["rgb"], r["depth"], r["sil"], rgb, depth, prior)
            b = oracle.backward(sc, oc, pose, op, L["d_rgb"], L["d_depth"], L["d_sil"])
            pose, state = oracle.adam_step(pose, state, b["pose6"], op)
        est_o.append(pose)
    el = time.perf_counter() - t0
    ce_g, ce_o = slam.camera_centres(np.array(est_gpu)), slam.camera_centres(np.array(est_o))
    dt = np.linalg.norm(ce_g - ce_o, axis=1)[1:]
    ang = []
    for a_, b_ in zip(est_gpu[1:], est_o[1:]):
        Ra, Rb = scenes.pose_rt(a_)[0], scenes.pose_rt(b_)[0]
        ang.append(float(np.degrees(np.arccos(np.clip((np.trace(Ra @ Rb.T) - 1) / 2, -1, 1)))))
    truth_o = _trajectory_report(np.array(est_o), np.array(poses))
    truth_g = _trajectory_report(np.array(est_gpu), np.array(poses))
    return {"workload": f"first {frames_n} frames of the spline path at 160x120, 200k room Gaussians (fp16), "
                        f"{iters} iterations per frame; the oracle on the same FP16-rounded attributes",
            "frames": frames_n, "trans_diff_mm_per_frame": [round(1e3 * float(x), 4) for x in dt],
            "rot_diff_deg_per_frame": [round(x, 5) for x in ang],
            "max_trans_diff_mm": round(1e3 * float(dt.max()), 4), "max_rot_diff_deg": round(max(ang), 5),
            "ate_vs_truth_cm": {"oracle": truth_o["ate_rmse_cm"], "gpu": truth_g["ate_rmse_cm"]},
            "oracle_seconds": round(el, 1)}


def accuracy_vs_oracle(dev, stream) -> dict:
    """Every timed workload's error against the FP64 oracle, on samples the oracle finishes
    on the host cores: the tracking frame, one batched view per resolution (BF16
    attributes: against the oracle on the dequantized attributes, and through the fused
    loss against the oracle on the FP32 attributes, the rounding of the storage included),
    one mapping keyframe (every parameter gradient), and the drift of the sequence tracker
    against the oracle's tracking loop."""
    import torch
    from paper_2408_05635_gb300 import scenes
    out = {}
    g, cam, gt_pose, start, rgb, depth, prior = workload()
    out["tracking_frame"], _ = _view_accuracy(dev, stream, g, g, cam, start, (rgb, depth, prior), torch.float32)
    gb, cams, poses0, frame_of, frames = batched_workload()
    gq = scenes.Gaussians(gb.means, *(torch.tensor(a).to(torch.bfloat16).float().numpy() for a in
                                      (gb.quats, gb.log_scales, gb.logits, gb.rgb)))
    views = {}
    for w in sorted({c.width for c in cams}):
        v = next(v for v, c in enumerate(cams) if c.width == w)
        res, fused_bf16 = _view_accuracy(dev, stream, gb, gq, cams[v], poses0[v], frames[frame_of[v]], torch.bfloat16)
        import oracle
        op = oracle.Params()
        sc32 = oracle.Scene(*gb.arrays())
        oc = oracle.camera(cams[v].fx, cams[v].fy, cams[v].cx, cams[v].cy, cams[v].width, cams[v].height)
        r32 = oracle.render(sc32, oc, poses0[v], op)
        L32 = oracle.loss(oc, op, r32["rgb"], r32["depth"], r32["sil"], *frames[frame_of[v]])
        o32 = oracle.backward(sc32, oc, poses0[v], op, L32["d_rgb"], L32["d_depth"], L32["d_sil"])
        res["bf16_pose_grad_vs_fp32_attribute_oracle_rel_err"] = _rel(fused_bf16, o32["pose6"])
        views[f"{cams[v].width}x{cams[v].height} (view {v})"] = res
    out["batched_bf16_views"] = views
    gm, mcams, mposes, mframes = mapping_workload()
    out["mapping_keyframe_1"], _ = _view_accuracy(dev, stream, gm, gm, mcams[1], mposes[1], mframes[1], torch.float32,
                                                  params_grads=True)
    out["sequence_drift"] = sequence_drift(dev, stream)
    return out


def oracle_small_single_thread(budget_s: float = 3.0) -> dict:
    """The oracle's tracking iteration on one host thread, on the small parity case
    (160 x 120, 2,000 Gaussians in front of the camera, target rendered 2 deg / 3 cm away,
    depth prior with 5 % holes), repeated until `budget_s` seconds have elapsed."""
    import oracle
    from paper_2408_05635_gb300 import scenes
    g, cam = scenes.cube_scene()
    threads_before = oracle.num_threads(oracle.Params())
    p = oracle.Params(n_threads=1)
    sc = oracle.Scene(*g.arrays())
    oc = oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)
    rng = np.random.default_rng(0)
    tgt = oracle.render(sc, oc, scenes.perturb_pose(scenes.identity_pose(), rng, 2.0, 0.03), p)
    prior = scenes.prior_from_depth(tgt["depth"], rng, 0.02, 0.05)
    pose, state = np.asarray(scenes.identity_pose(), np.float64).copy(), np.zeros(16)
    iters, t0 = 0, time.perf_counter()
    while True:
        r = oracle.render(sc, oc, pose, p)
        L = oracle.loss(oc, p, r["rgb"], r["depth"], r["sil"], tgt["rgb"], tgt["depth"], prior)
        b = oracle.backward(sc, oc, pose, p, L["d_rgb"], L["d_depth"], L["d_sil"])
        pose, state = oracle.adam_step(pose, state, b["pose6"], p)
        iters += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    its = iters / el
    cores = oracle.num_threads(p)
    oracle.num_threads(oracle.Params(n_threads=threads_before))  # the oracle's thread count as it was
    return {"value": its * cam.width * cam.height / 1e6, "unit": "Mpix/s", "iters_per_s": its, "cores": cores,
            "sample": f"{iters} full tracking iterations of the 160x120 / 2k case in {el:.1f} s"}


def ncu_traffic(kernel):
    """(DRAM bytes per launch of `kernel` from the committed ncu summary, or None once the
    kernel's sources differ from the ones the counters were taken on; the summary's path)."""
    import glob
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    for path in sorted(glob.glob(os.path.join(root, "profiles", "*.md"))):
        for line in open(path):
            f = line.split()
            if len(f) >= 5 and f[0] == "traffic" and f[1] == kernel:
                h = hashlib.sha256()
                for src in f[4:]:
                    h.update(open(os.path.join(root, "paper_2408_05635_gb300", "csrc", src), "rb").read())
                return (int(f[2]) if h.hexdigest()[:16] == f[3] else None), os.path.relpath(path, root)
    return None, None


def reference_steps(g, cam, start, rgb, depth, prior, steps: int, warmup: int, band: int = 64):
    """Seconds of each timed oracle step: one full FP64 tracking iteration (render, loss,
    backward, decoupled Adam) on a `band`-row band of the frame.  The bands step down the
    frame and wrap around within it, so every band lies wholly inside the image."""
    import oracle
    p = oracle.Params()
    sc = oracle.Scene(*g.arrays())
    H, W = cam.height, cam.width
    band = min(band, H)
    nbands = H // band
    times = []
    pose, state = np.asarray(start, np.float64).copy(), np.zeros(16)
    for it in range(warmup + steps):
        y0 = (it % nbands) * band
        sub = oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy - y0, W, band)
        sl = slice(y0, y0 + band)
        t0 = time.perf_counter()
        r = oracle.render(sc, sub, pose, p)
        L = oracle.loss(sub, p, r["rgb"], r["depth"], r["sil"], rgb[:, sl], depth[sl], prior[sl])
        b = oracle.backward(sc, sub, pose, p, L["d_rgb"], L["d_depth"], L["d_sil"])
        pose, state = oracle.adam_step(pose, state, b["pose6"], p)
        dt = time.perf_counter() - t0
        if it >= warmup:
            times.append(dt)
    return times, oracle.num_threads(p)


def run_reference(a, rank, world):
    if rank != 0:
        return
    g, cam, gt, start, rgb, depth, prior = workload()
    W, band = cam.width, 64
    times, cores = reference_steps(g, cam, start, rgb, depth, prior, a.steps, a.warmup, band)
    total = sum(times)
    mpix = a.steps * W * band / total / 1e6
    sample = f"each step: one full oracle tracking iteration on a {W}x{band} band of the 640x480 / 200k frame"
    line = {"impl": "reference", "metric": METRIC, "value": mpix, "unit": "Mpix/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": mpix, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mpix, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sm_count() -> int:
    """Streaming multiprocessors of the current GPU, read from the device."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def hbm_peak_gbs() -> tuple[float, str]:
    """Measured HBM copy bandwidth of this GPU type (MEASURED_PEAKS.json), else the
    fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_rooflines(kern_ms: dict, n_gauss: int, views: int, attr_bytes: int, records: int, pairs: int,
                     fwd_contrib: int, bwd_contrib: int, mhz: float, n_sm: int | None = None,
                     radix_passes: int = 6) -> dict:
    """Every kernel of a tracking iteration against the roofline that bounds it: its
    algorithmic bytes or FLOPs per launch (from the work counted on the device) over its
    CUDA-event time (markers around every kernel, so each time includes its launch gap),
    as a fraction of the measured HBM copy bandwidth or of the FP32 FMA peak at the
    sampled SM clock.  k_scan_tiles (one block) and k_finalize (a chain of dependent
    steps) are latency-bound: their times are reported without a roofline."""
    hbm, hbm_from = hbm_peak_gbs()
    n_sm = n_sm or sm_count()
    fp32 = n_sm * FP32_LANES * 2 * mhz * 1e6 / 1e12
    work = {
        "k_project": ("hbm", 12 * n_gauss * views + (attr_bytes + 96) * records,
                      f"12 B of means per (Gaussian, view); {attr_bytes} B of other parameters and a 96 B record "
                      "per visible (Gaussian, view)"),
        "k_emit": ("hbm", 12 * pairs, "12 B per (Gaussian, tile) pair"),
        "k_forward": ("alu", FLOP_FWD_PAIR * fwd_contrib, f"{FLOP_FWD_PAIR} FLOP per contributing pair"),
        "k_backward": ("alu", FLOP_BWD_PAIR * bwd_contrib, f"{FLOP_BWD_PAIR} FLOP per differentiated pair"),
        "k_track_tile": ("alu", FLOP_FWD_PAIR * fwd_contrib + FLOP_BWD_PAIR * bwd_contrib,
                         f"{FLOP_FWD_PAIR} FLOP per contributing and {FLOP_BWD_PAIR} per differentiated pair"),
        "k_radix_sort": ("hbm", 24 * radix_passes * pairs,
                         f"{radix_passes} passes x 24 B per (Gaussian, tile) pair (key and value read and written)"),
        "k_bproject": ("alu", FLOP_BPROJ_REC * records, f"about {FLOP_BPROJ_REC} FLOP per record"),
    }
    out = {}
    for k, ms in kern_ms.items():
        if k not in work or ms <= 0:
            out[k] = {"bound": "latency", "us": round(1e3 * ms, 2)}
            continue
        bound, units, what = work[k]
        if bound == "hbm":
            achieved, peak, unit = units / (ms / 1e3) / 1e9, hbm, "GB/s"
        else:
            achieved, peak, unit = units / (ms / 1e3) / 1e12, fp32, "TFLOP/s"
        out[k] = {"bound": bound, "us": round(1e3 * ms, 2), "achieved": float(f"{achieved:.4g}"),
                  "peak": round(peak, 1), "unit": unit, "frac": float(f"{achieved / peak:.3g}"), "work": what}
    out["peaks_from"] = f"HBM {hbm:.0f} GB/s ({hbm_from}); FP32 {fp32:.1f} TFLOP/s ({n_sm} SMs at {mhz:.0f} MHz)"
    return out


def max_over_ranks(value: float, world: int, device) -> float:
    """The largest of every rank's value (the slowest replica sets the job's time); the
    plain value with one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: float, steps: int, world: int, ms_max: float) -> float:
    """Units all ranks processed per second: every replica does `steps` steps of
    `units_per_step` units, and the job takes the slowest replica's time (weak scaling)."""
    return world * steps * units_per_step / (ms_max / 1e3)


def main():
    a = _args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    import torch
    import torch.distributed as dist
    from paper_2408_05635_gb300 import gs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    g, cam, gt_pose, start, rgb, depth, prior = workload(seed=rank)
    R = gs.Rasterizer(gs.Config(), device=dev)
    gt = gs.GaussianTensors.from_numpy(g, device=dev)
    # the step's result (pose, then the loss) in one 8-double buffer, and the frame's three
    # planes in one float buffer, so the end-to-end leg moves each with a single copy
    out8 = torch.zeros(8, dtype=torch.float64, device=dev)
    poses = out8[:7].view(1, 7)
    poses.copy_(torch.tensor(np.asarray(start)[None], dtype=torch.float64))
    loss = out8[7:].view(1, 1)
    P_px = cam.width * cam.height
    frame_dev = torch.tensor(np.concatenate([rgb.reshape(-1), depth.reshape(-1), prior.reshape(-1)]), device=dev)
    t_rgb, t_depth, t_prior = frame_dev[:3 * P_px], frame_dev[3 * P_px:4 * P_px], frame_dev[4 * P_px:]
    targets = gs.gs_targets(t_rgb.data_ptr(), t_depth.data_ptr(), t_prior.data_ptr())
    sched = apply_schedule(a, R, [cam], gt, poses, (t_rgb, t_depth, t_prior))
    prob = R.plan(gt, [cam], poses, margin=1.5)
    ws, nb = R.workspace(prob)
    adam = torch.zeros(1, 16, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step():
        gs.gs_track_step(R.ctx, prob, gt.c(), targets, poses, adam, loss, 1, ws, nb, stream)

    for _ in range(a.warmup):
        step()
    # per-kernel breakdown (CUDA-event markers between all of the library's kernels, which
    # cost a few microseconds each); it also names the dominant kernel
    gs.gs_set_profiling(R.ctx, True)
    start_pose = torch.tensor(np.asarray(start)[None], dtype=torch.float64, device=dev)
    breakdown, n_break = {}, min(a.steps, 200)
    for k in range(n_break):
        if k % ITERS_PER_FRAME == 0:
            poses.copy_(start_pose)
            adam.zero_()
        flush.fill_(float(k))
        step()
        for name, ms in gs.gs_kernel_times(R.ctx):
            breakdown[name] = breakdown.get(name, 0.0) + ms
    breakdown = {k: v / n_break for k, v in breakdown.items()}
    dominant = max(breakdown, key=breakdown.get)
    # timed steps: markers around the dominant kernel only
    gs.gs_set_profiling_mask(R.ctx, [dominant])
    step()
    poses.copy_(start_pose)
    adam.zero_()
    counts = R.sync(stream)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    kern_ms, contrib = {}, {"fwd_evals": 0, "fwd_contrib": 0, "bwd_evals": 0, "bwd_contrib": 0}
    launches = 0
    # the view-table copy, the projection, scan and emission, the compositing (two kernels,
    # or one fused), the back-projection and the finalize
    sch = R.schedule
    tiles = -(-cam.width // sch["tile_w"]) * -(-cam.height // sch["tile_h"])
    radix = 3 * gs.radix_passes(tiles) + 1 if sch["flags"] & gs.GS_SCHED_RADIX else 0  # passes x 3 + ties
    per_iter_launches = 1 + 3 + radix + (1 if sch["flags"] & gs.GS_SCHED_FUSED else 2) + 2
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(a.steps):
            if k % ITERS_PER_FRAME == 0:  # a new frame: tracking restarts from the start pose
                poses.copy_(start_pose)
                adam.zero_()
            flush.fill_(float(k))
            starts[k].record(stream)
            step()
            ends[k].record(stream)
            kt = gs.gs_kernel_times(R.ctx)  # waits for this step's markers
            for name, ms in kt:
                kern_ms[name] = kern_ms.get(name, 0.0) + ms
            launches += per_iter_launches
            st_k, c_k = gs.gs_sync_status(R.ctx, stream)
            for key in contrib:
                contrib[key] += getattr(c_k, key)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    gs.gs_set_profiling(R.ctx, False)
    st, c = gs.gs_sync_status(R.ctx, stream)
    if st:
        raise SystemExit(f"device reported {gs._STATUS[st]} during the timed steps")
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_max = max_over_ranks(ms, world, dev)
    pix = cam.width * cam.height
    iters_per_s = whole_job_rate(1, a.steps, world, ms_max)
    mpix = iters_per_s * pix / 1e6

    # end to end through the public call with host buffers: the pinned frame in (read in
    # place by the kernels over the coherent host link, or copied by gs_track_step_upload
    # into the device targets beside the iteration's binning), pose and loss out (stored
    # into pinned host memory by the last kernel)
    h_frame = torch.tensor(np.concatenate([rgb.reshape(-1), depth.reshape(-1), prior.reshape(-1)])).pin_memory()
    h_out = torch.empty(8, dtype=torch.float64).pin_memory()
    src = gs.gs_host_targets(h_frame[:3 * P_px].data_ptr(), h_frame[3 * P_px:4 * P_px].data_ptr(),
                             h_frame[4 * P_px:].data_ptr(), h_out.data_ptr())

    def e2e_run(dev_targets):
        e2e_s, e2e_e = [], []
        for k in range(a.warmup + a.steps):
            if k % ITERS_PER_FRAME == 0:
                poses.copy_(start_pose)
                adam.zero_()
            flush.fill_(float(k))
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            # the frame in, and the pose and loss out: the finalize kernel stores them into h_out
            gs.gs_track_step_upload(R.ctx, prob, gt.c(), dev_targets, src, poses, adam, loss, 1, ws, nb, stream)
            s1.record(stream)
            if k >= a.warmup:
                e2e_s.append(s0)
                e2e_e.append(s1)
        torch.cuda.synchronize(dev)
        e2e_ms = sum(s.elapsed_time(e) for s, e in zip(e2e_s, e2e_e))
        return whole_job_rate(pix, a.steps, world, max_over_ranks(e2e_ms, world, dev)) / 1e6

    e2e_mpix = e2e_run(None)              # read in place
    e2e_copy_mpix = e2e_run(targets)      # copied into the device targets

    # roofline of the dominant kernel, from its CUDA-event time inside the timed steps
    avg = {k: v / a.steps for k, v in kern_ms.items()}
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz") or 2070.0
    n_sm = sm_count()
    peak_tflops = n_sm * FP32_LANES * 2 * mhz * 1e6 / 1e12
    per_pair = {"k_backward": (FLOP_BWD_PAIR, contrib["bwd_contrib"], f"{FLOP_BWD_PAIR} FP32 FLOP per differentiated "
                                                                       "(pixel, Gaussian) pair"),
                "k_forward": (FLOP_FWD_PAIR, contrib["fwd_contrib"], f"{FLOP_FWD_PAIR} FP32 FLOP per contributing "
                                                                     "(pixel, Gaussian) pair"),
                "k_track_tile": (1, FLOP_FWD_PAIR * contrib["fwd_contrib"] + FLOP_BWD_PAIR * contrib["bwd_contrib"],
                                 f"{FLOP_FWD_PAIR} FP32 FLOP per contributing and {FLOP_BWD_PAIR} per differentiated "
                                 "(pixel, Gaussian) pair")}
    roofline = None
    if dominant in per_pair:
        f, units, what = per_pair[dominant]
        achieved = f * units / a.steps / (avg[dominant] / 1e3) / 1e12
        traffic, traffic_src = ncu_traffic(dominant)
        roofline = {"kernel": dominant, "bound": "alu", "achieved": achieved, "peak": peak_tflops,
                    "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                    "traffic_from": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, cold cache "
                                    f"({traffic_src})",
                    "work": f"{what}: {f * units // a.steps} FLOP per launch",
                    "peak_from": f"{n_sm} SMs x {FP32_LANES} FP32 lanes x 2 x {mhz:.0f} MHz (median SM clock, timed region)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": mpix, "unit": "Mpix/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (room scene; ray-cast RGB-D frame)",
            "config": {"workload": WORKLOAD, "width": cam.width, "height": cam.height, "gaussians": N_GAUSS,
                       "pairs": int(counts.n_pairs), "records": int(counts.n_records),
                       "max_tile_pairs": int(counts.max_tile),
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}",
                       "launch_schedule": sched},
            "tracking_iters_per_s": iters_per_s,
            "e2e": {"value": e2e_mpix, "unit": "Mpix/s",
                    "h2d_bytes_per_step": int(h_frame.numel() * h_frame.element_size()),
                    "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size()),
                    "frame": "page-locked host memory read in place by the kernels (coherent host link)",
                    "copied_upload": {"value": e2e_copy_mpix, "unit": "Mpix/s",
                                      "frame": "copied into device targets beside the binning"}},
            "gpu_launches": launches,
            "clocks": clocks,
            "roofline": roofline,
            "kernels_us": {k: round(1e3 * v, 2) for k, v in sorted(breakdown.items(), key=lambda kv: -kv[1])},
            "kernels_us_note": f"{n_break} steps with event markers around every kernel (event nodes on a side "
                               f"branch of the graph; a kernel's time runs from the previous kernel's end marker "
                               f"to its own, launch gap included); the timed steps mark only {dominant}",
            "pairs_per_step": {k: v // a.steps for k, v in contrib.items()},
            # (pixel, Gaussian) pairs that contributed to Eqs. 2-4 or were differentiated, per second
            "useful_pair_evals_per_s": (contrib["fwd_contrib"] + contrib["bwd_contrib"]) / (ms / 1e3),
            "roofline_kernels": kernel_rooflines(breakdown, N_GAUSS, 1, 44, int(counts.n_records), int(counts.n_pairs),
                                                 contrib["fwd_contrib"] // a.steps, contrib["bwd_contrib"] // a.steps,
                                                 mhz),
        }
        if world == 1 and a.isotropic_steps > 0:
            line["isotropic"] = run_isotropic(dev, stream, a.isotropic_steps)
        if world == 1 and a.batched_steps > 0:
            line["batched"] = run_batched(a, dev, stream, mhz)
        if world == 1 and a.mapping_steps > 0:
            line["mapping"] = run_mapping(a, dev, stream)
        if world == 1 and a.sequence_frames > 0:
            line["sequence"] = run_sequence(a, dev, stream)
        if world == 1 and not a.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g, cam, start, rgb, depth, prior, a.cpu_sample_seconds)
            line["cpu_baseline"]["single_thread_small_case"] = oracle_small_single_thread()
            # the oracle run of the CPU-baseline leg also gives every timed workload's error
            # against FP64
            t0 = time.perf_counter()
            line["cpu_baseline"]["accuracy_vs_oracle"] = accuracy_vs_oracle(dev, stream)
            line["cpu_baseline"]["accuracy_vs_oracle"]["seconds"] = round(time.perf_counter() - t0, 1)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
