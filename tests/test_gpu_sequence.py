"""Sequences: frame-to-frame tracking (slam.Tracker: gs_track_step over every frame,
started from the previous estimate) against the oracle's tracking loop, and the whole
loop of Sec. III (slam.Slam) on a short sequence from an empty map.

Tolerance of the trajectory parity: Adam moves each pose coordinate by at most lr per
iteration, so a sign flip of a near-zero gradient component costs at most 2 lr; the
bound is 4 lr per frame, and the measured gap is printed.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import ocam
from paper_2408_05635_gb300 import gs, scenes, slam

pytestmark = pytest.mark.gpu

CAM = scenes.Cam(262.5, 262.5, 159.5, 119.5, 320, 240)


def _pose_gap(a, b):
    from scipy.spatial.transform import Rotation
    Ra, ta = scenes.pose_rt(a)
    Rb, tb = scenes.pose_rt(b)
    return (float(np.linalg.norm(-Ra.T @ ta + Rb.T @ tb)),
            float(np.linalg.norm(Rotation.from_matrix(Ra @ Rb.T).as_rotvec())))


def test_frame_to_frame_tracking_follows_oracle():
    """Four frames of the long sequence's path (about 4 cm and 2 deg apart), 12 iterations
    each on a 30k-Gaussian room, every frame started from the previous estimate (each side
    its own), with the depth prior.  The loss histories agree on the first frame (same
    start); afterwards the starts differ by the previous frames' gaps."""
    g = scenes.room_scene(30_000, seed=1)
    poses = scenes.spline_trajectory(200, seed=1)[:4]
    rng = np.random.default_rng(3)
    frames = []
    for p in poses:
        rgb, depth = scenes.raycast_room(p, CAM, seed=1)
        frames.append((np.ascontiguousarray(rgb), np.ascontiguousarray(depth), scenes.prior_from_depth(depth, rng, 0.02, 0.05)))
    iters = 12
    op = oracle.Params()
    sc, oc = oracle.Scene(*g.arrays()), ocam(CAM)
    tr = slam.Tracker(CAM, iters)
    gt = gs.GaussianTensors.from_numpy(g)
    est = torch.tensor(poses[0], dtype=torch.float64, device="cuda")
    o_pose = np.asarray(poses[0], np.float64)
    gaps = []
    for k in range(1, len(poses)):
        rgb, depth, prior = (torch.from_numpy(x).cuda() for x in frames[k])
        est = tr.track(gt, est, rgb, depth, prior)
        losses = []
        state = np.zeros(16)
        for _ in range(iters):
            r = oracle.render(sc, oc, o_pose, op)
            L = oracle.loss(oc, op, r["rgb"], r["depth"], r["sil"], *frames[k])
            losses.append(L["loss"])
            b = oracle.backward(sc, oc, o_pose, op, L["d_rgb"], L["d_depth"], L["d_sil"])
            o_pose, state = oracle.adam_step(o_pose, state, b["pose6"], op)
        if k == 1:
            np.testing.assert_allclose(tr.hist.cpu().numpy()[:, 0], losses, rtol=5e-3)
        gaps.append(_pose_gap(est.cpu().numpy(), o_pose))
        gt_gap = _pose_gap(o_pose, poses[k])
        print(f"frame {k}: GPU-oracle gap {gaps[-1][0]:.2e} m {gaps[-1][1]:.2e} rad; oracle vs truth {gt_gap[0]:.3f} m")
        assert gaps[-1][0] < 4 * op.lr_trans * k and gaps[-1][1] < 4 * op.lr_rot * k
    tr.close()


@pytest.mark.parametrize("iso", [False, True])
def test_slam_loop_builds_a_map_and_tracks(iso):
    """Sec. III on the first 13 frames of the long sequence's path (QVGA): first-frame
    Gaussians, tracking, keyframes every 4 frames with silhouette-driven additions, 30
    mapping iterations per keyframe (100 on the first), removal; with anisotropic
    Gaussians and with the isotropic ones of Eq. 1.  The trajectory stays within a few cm
    of the truth, the map grows on the keyframes and renders the keyframes back
    recognisably."""
    poses = scenes.spline_trajectory(200, seed=2)[:13]
    frames = []
    for p in poses:
        rgb, depth = scenes.raycast_room_torch(p, CAM, seed=2, device="cuda")
        frames.append((rgb, depth, None))
    cfg = slam.SlamConfig(capacity=400_000, lowp=torch.float16, isotropic=iso)
    S = slam.Slam(CAM, cfg)
    for k in range(len(poses)):
        S.process(k, *frames[k], first_pose=poses[0] if k == 0 else None)
    est = torch.stack(S.poses).cpu().numpy()
    d = np.linalg.norm(slam.camera_centres(est) - slam.camera_centres(poses), axis=1)
    q = S.evaluate(frames)
    print(f"ATE {100 * np.sqrt(np.mean(d * d)):.2f} cm, max {100 * d.max():.2f} cm, map {S.n}, "
          f"added {S.stats['added']}, pruned {S.stats['pruned']}, quality {q}")
    assert S.stats["keyframes"] == 4
    assert all(a > 0 for a in S.stats["added"])
    assert d.max() < 0.05
    assert q["psnr_db"] > 20.0 and q["depth_l1_cm"] < 5.0
    S.close()
