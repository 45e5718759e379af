"""Frame-by-frame driver of the method's three steps (Sec. III): the first frame's
Gaussians (Sec. III-A), tracking of every frame against the fixed map (Sec. III-B) and,
on keyframes, new Gaussians where the silhouette shows new observations followed by
gradient-based optimisation of the map over a window of keyframes with their poses fixed
and the removal of Gaussians whose opacity fell away (Sec. III-C).

Host code here only sequences calls into the CUDA library (gs.py): every computation on
images, Gaussians and poses runs in its kernels.  Per frame the host waits once, to read
the device status (a pair-capacity overflow re-plans the frame and tracks it again);
on a keyframe it also reads the live Gaussian count.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import gs

@dataclasses.dataclass
class SlamConfig:
    """Readings where the paper is silent (its keyframes follow feature parallax, which a
    synthetic sequence has no features for)."""
    track_iters: int = 100        # tracking iterations per frame, one CUDA graph
    keyframe_every: int = 4       # every k-th frame is a keyframe
    window: int = 64              # the most recent keyframes optimised together
    map_iters: int = 30           # mapping iterations per keyframe (Adam moments reset per keyframe)
    first_map_iters: int = 100    # on the first frame, whose half-opaque one-pixel Gaussians
                                  # leave few pixels above the tracking mask's S > 0.99
    map_chunk: int = 8            # views per mapping call
    plan_margin: float = 1.5      # pair capacity over the pairs measured when planning
    lowp: torch.dtype | None = None  # track on a BF16 / F16 render copy of the map
    capacity: int = 4_000_000     # Gaussians the map can hold
    prune: bool = True            # remove Gaussians with opacity < opacity_min after mapping
    isotropic: bool = False       # Eq. 1 as written: no rotation, one radius per Gaussian
    autotune_reps: int = 0        # > 0: the tracker tunes its launch schedule (gs_autotune,
                                  # that many passes per setting) on the first frame and
                                  # again whenever the map has doubled since


class Tracker:
    """Tracking with the map fixed (Sec. III-B): `iters` decoupled rotation / translation
    iterations in one gs_track_step call (one CUDA graph), starting from a given pose
    (the previous frame's estimate in a sequence).  The frame is copied into fixed device
    buffers so the graph is reused from frame to frame.  With autotune_reps > 0 the launch
    schedule is tuned on the first frame and re-tuned when the map has doubled."""

    def __init__(self, cam, iters: int, config: gs.Config | None = None, device="cuda", margin: float = 1.5,
                 autotune_reps: int = 0):
        self.cam, self.iters, self.margin = cam, int(iters), margin
        self.autotune_reps = int(autotune_reps)
        self.tuned_n, self.tune, self.tunes = None, None, 0
        self.dev = torch.device(device)
        self.R = gs.Rasterizer(config or gs.Config(), device)
        P = int(cam.width) * int(cam.height)
        self.t_rgb = torch.zeros(3 * P, dtype=torch.float32, device=device)
        self.t_depth = torch.zeros(P, dtype=torch.float32, device=device)
        self.t_prior = torch.zeros(P, dtype=torch.float32, device=device)
        self.pose = torch.zeros(1, 7, dtype=torch.float64, device=device)
        self.adam = torch.zeros(1, 16, dtype=torch.float64, device=device)
        self.hist = torch.zeros(self.iters, 1, dtype=torch.float64, device=device)
        self.prob, self.key = None, None
        self.replans = 0

    def close(self):
        self.R.close()

    def track(self, g: gs.GaussianTensors, start: torch.Tensor, rgb, depth, prior=None, stream=None) -> torch.Tensor:
        """Pose (device, 7 doubles) after the iterations; the loss history is in self.hist."""
        self.t_rgb.copy_(rgb.reshape(-1), non_blocking=True)
        self.t_depth.copy_(depth.reshape(-1), non_blocking=True)
        has_prior = prior is not None
        if has_prior:
            self.t_prior.copy_(prior.reshape(-1), non_blocking=True)
        tg = gs.gs_targets(self.t_rgb.data_ptr(), self.t_depth.data_ptr(), self.t_prior.data_ptr() if has_prior else None)
        key = (g.means.data_ptr(), g.n, g.log_scales.dtype, g.isotropic)
        for _ in range(4):
            self.pose.copy_(start.reshape(1, 7))
            self.adam.zero_()
            if self.prob is None or key != self.key:
                if self.autotune_reps > 0 and (self.tuned_n is None or g.n > 2 * self.tuned_n):
                    # tuned on a problem with twice the pair margin, so that the smaller
                    # tiles (more pairs) are timed too
                    tprob = self.R.plan(g, [self.cam], self.pose, margin=2 * self.margin)
                    tgt = (self.t_rgb, self.t_depth, self.t_prior if has_prior else None)
                    self.tune = self.R.autotune(tprob, g, self.pose, tgt, pose_only=True, reps=self.autotune_reps,
                                                stream=stream)
                    self.tuned_n = g.n
                    self.tunes += 1
                self.prob = self.R.plan(g, [self.cam], self.pose, margin=self.margin)
                self.key = key
            ws, nb = self.R.workspace(self.prob)
            gs.gs_track_step(self.R.ctx, self.prob, g.c(), tg, self.pose, self.adam, self.hist, self.iters, ws, nb,
                             stream)
            st, counts = gs.gs_sync_status(self.R.ctx, stream)
            if st == 0:
                return self.pose[0].clone()
            if st != gs.GS_ERR_CAPACITY:
                raise gs.GsError(st, "tracking")
            # the camera moved to where more (Gaussian, tile) pairs are visible: re-plan
            need = max(int(counts.n_pairs), 2 * int(self.prob.pair_capacity))
            self.prob = self.R.problem(g.n, [self.cam], int(need * self.margin) + 1024)
            self.replans += 1
        raise RuntimeError("tracking: pair capacity kept overflowing")


class Slam:
    """The whole loop on one RGB-D sequence (Sec. III).  Frames are given as device
    tensors (rgb 3 x H x W, depth H x W, prior H x W or None); the first frame's pose fixes
    the world frame (the paper takes the identity)."""

    def __init__(self, cam, cfg: SlamConfig | None = None, device="cuda", config: gs.Config | None = None):
        self.cam, self.cfg = cam, cfg or SlamConfig()
        self.dev = torch.device(device)
        c = self.cfg
        self.map = gs.Map(c.capacity, device, lowp_dtype=c.lowp, isotropic=c.isotropic)
        self.spare = gs.Map(c.capacity, device, lowp_dtype=c.lowp, isotropic=c.isotropic) if c.prune else None
        self.tracker = Tracker(cam, c.track_iters, config, device, c.plan_margin, c.autotune_reps)
        self.mapper = gs.Rasterizer(config or gs.Config(), device)
        self.grads = {k: torch.zeros_like(self.map.p[k]) for k in self.map.GROUPS}
        self.keyframes: list[tuple[torch.Tensor, tuple]] = []
        self.poses: list[torch.Tensor] = []
        self.n = 0
        self.stats = {"keyframes": 0, "added": [], "pruned": [], "map_size": []}

    def close(self):
        self.tracker.close()
        self.mapper.close()

    def gaussians(self, lowp: bool | None = None) -> gs.GaussianTensors:
        lowp = self.cfg.lowp is not None if lowp is None else lowp
        return self.map.gaussians(self.n, lowp=lowp)

    def process(self, k: int, rgb, depth, prior=None, first_pose=None, stream=None) -> torch.Tensor:
        """One frame: initialise (k = 0) or track; on keyframes add Gaussians and optimise
        the map.  Returns the frame's pose (device, 7 doubles)."""
        if k == 0:
            pose = torch.as_tensor(np.asarray(first_pose, np.float64), device=self.dev).reshape(7).contiguous()
            self.map.add_from_frame(self.cam, pose, rgb, depth, None, stream)
            keyframe = True
        else:
            pose = self.tracker.track(self.gaussians(), self.poses[-1], rgb, depth, prior, stream)
            keyframe = k % self.cfg.keyframe_every == 0
            if keyframe:
                # the silhouette at the tracked pose marks what the map already explains
                g = self.gaussians(lowp=False)
                prob = self.mapper.plan(g, [self.cam], pose.reshape(1, 7), margin=self.cfg.plan_margin)
                out = self.mapper.render(prob, g, pose.reshape(1, 7), stream=stream)
                self.mapper.sync(stream)
                self.map.add_from_frame(self.cam, pose, rgb, depth, out["sil"], stream)
        self.poses.append(pose)
        if keyframe:
            n_before = self.n
            self.n = self.map.n
            self.stats["added"].append(self.n - n_before)
            self.keyframes.append((pose.clone(), (rgb, depth, prior)))
            self.optimise_map(stream)
            self.stats["keyframes"] += 1
            self.stats["map_size"].append(self.n)
        return pose

    def optimise_map(self, stream=None) -> None:
        """map_iters Adam steps on the map over the most recent `window` keyframes."""
        c = self.cfg
        win = self.keyframes[-c.window:]
        cams = [self.cam] * len(win)
        poses = torch.stack([p for p, _ in win]).contiguous()
        targets = [t for _, t in win]
        n = self.n
        g = self.map.gaussians(n, lowp=False)
        probs = [self.mapper.plan(g, cams[v0:v0 + c.map_chunk], poses[v0:v0 + c.map_chunk].contiguous(),
                                  margin=c.plan_margin) for v0 in range(0, len(win), c.map_chunk)]
        views = {k: self.grads[k][:n] for k in self.map.GROUPS}
        self.map.state.zero_()
        iters = c.first_map_iters if len(self.keyframes) == 1 else c.map_iters
        for it in range(1, iters + 1):
            for t in views.values():
                t.zero_()
            self.mapper.mapping_grads(g, cams, poses, targets, chunk=c.map_chunk, grads=views, probs=probs,
                                      stream=stream)
            self.map.adam_step(self.grads, it, stream)
        self.mapper.sync(stream)
        if c.prune:
            self.map.prune_into(self.spare, stream)
            self.map, self.spare = self.spare, self.map
            n_new = self.map.n
            self.stats["pruned"].append(n - n_new)
            self.n = n_new

    def evaluate(self, frames, stream=None) -> dict:
        """Image quality of the final map at the keyframes' estimated poses (Sec. IV:
        PSNR of the colour, average depth error): gs_image_metrics per keyframe."""
        g = self.gaussians(lowp=False)
        W, H = int(self.cam.width), int(self.cam.height)
        ssim_ok = min(W, H) >= 176  # the coarsest of the five scales must hold one window
        sums = torch.zeros(len(self.keyframes), 4, dtype=torch.float64, device=self.dev)
        ssim = torch.zeros(len(self.keyframes), 4, dtype=torch.float64, device=self.dev)
        for j, (pose, (rgb, depth, _)) in enumerate(self.keyframes):
            prob = self.mapper.plan(g, [self.cam], pose.reshape(1, 7), margin=self.cfg.plan_margin)
            out = self.mapper.render(prob, g, pose.reshape(1, 7), stream=stream)
            gs.gs_image_metrics(out["rgb"], out["depth"], rgb.reshape(-1), depth.reshape(-1), sums[j], stream)
            if ssim_ok:
                gs.gs_msssim(out["rgb"], rgb.reshape(-1), W, H, ssim[j], stream)
        self.mapper.sync(stream)
        s = sums.cpu().numpy()
        mse = s[:, 0] / (3 * W * H)
        res = {"psnr_db": float(np.mean(10 * np.log10(1.0 / np.maximum(mse, 1e-30)))),
               "depth_l1_cm": float(100 * s[:, 1].sum() / max(s[:, 2].sum(), 1.0)),
               "depth_rmse_cm": float(100 * np.sqrt(s[:, 3].sum() / max(s[:, 2].sum(), 1.0)))}
        if ssim_ok:
            res["ms_ssim"] = float(ssim[:, 0].mean().item())
        return res


def camera_centres(poses) -> np.ndarray:
    """World positions -R^T t of world->camera poses (n x 7)."""
    p = np.asarray(poses, np.float64).reshape(-1, 7)
    q = p[:, :4] / np.linalg.norm(p[:, :4], axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    return -np.einsum("nji,nj->ni", R, p[:, 4:7])
