"""Launch schedules through the C ABI (gs_set_schedule, gs_autotune).

The tile shape (and with it the threads per tile), the sub-buckets per tile and the
compositors' batch depths change how the work is launched, not what is computed.  With
the tile shape fixed, every schedule renders the same images bit for bit (each pixel
composites the same Gaussians in the same order, Eqs. 2-4, from the same tile-relative
coordinates) and the same gradients up to FP32 summation order.  Another tile shape
moves the tile origins the footprints are evaluated from, which changes their rounding:
images then agree to 2e-6 on the pixels the oracle marks unambiguous (a pixel where an
alpha_min or t_min decision sits within rounding of its threshold may take the other
branch).  Every schedule stays within the oracle tolerances (images 1e-4 on unambiguous
pixels, gradients 1e-3 relative).  The scene puts a few hundred Gaussians on the tiles of a ragged 75 x 53
image, so every schedule below takes several batches on its fullest tile (counted
exactly on the CPU from the oracle's footprints: 409 for 16 x 16 tiles, 426 for 32 x 8,
280 for 16 x 8, 175 for 8 x 8, 445 for 8 x 32, 319 for 32 x 4).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import assert_grads_close, assert_images_close, ocam, params_pair, rel_err
from paper_2408_05635_gb300 import gs, scenes, slam

pytestmark = pytest.mark.gpu

# (tile_w, tile_h, sub_buckets, fwd_batch, bwd_batch)
SCHEDULES = [(16, 16, 4, 256, 256), (16, 16, 1, 64, 64), (16, 16, 2, 128, 128), (16, 16, 4, 64, 256),
             (32, 8, 2, 256, 64), (16, 8, 4, 128, 64), (8, 8, 1, 64, 64), (8, 32, 4, 256, 128),
             (32, 4, 2, 128, 128)]
GRAD_KEYS = [("means", 0, 3), ("quats", 3, 7), ("log_scales", 7, 10), ("logits", 10, 11), ("rgb", 11, 14)]
NAMES = ("tile_w", "tile_h", "sub_buckets", "fwd_batch", "bwd_batch", "flags")
DEFAULT = dict(zip(NAMES, (16, 16, 4, 256, 256, 0)))


@pytest.fixture(scope="module")
def case():
    g, _ = scenes.cube_scene(n=4000, seed=11)
    cam = scenes.Cam(70.0, 72.0, 37.3, 27.1, 75, 53)
    pose = scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(3), 1.0, 0.02)
    gcfg, op = params_pair()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    ref = oracle.render(sc, oc, pose, op)
    H, W = cam.height, cam.width
    amb = ref["amb"]
    rng = np.random.default_rng(4)
    up = [np.where(amb[None], 0.0, rng.normal(size=(3, H, W))), np.where(amb, 0.0, rng.normal(size=(H, W))),
          np.where(amb, 0.0, rng.normal(size=(H, W)))]
    ob = oracle.backward(sc, oc, pose, op, *up)
    return g, cam, pose, gcfg, ref, up, ob


def _same_images(out, base, same_tile, amb, H, W):
    """Bit for bit with the default run when the tile shape is the same; else to 2e-6 on
    unambiguous pixels."""
    for k, ch in (("rgb", 3), ("depth", 1), ("sil", 1)):
        if same_tile:
            np.testing.assert_array_equal(out[k], base[k], err_msg=k)
        else:
            d = np.abs(out[k].reshape(ch, H, W) - base[k].reshape(ch, H, W)).max(axis=0)
            assert d[~amb].max() <= 2e-6, (k, d[~amb].max())


def _run(R, g, cam, pose, up):
    gt = gs.GaussianTensors.from_numpy(g)
    poses = torch.tensor(np.asarray(pose)[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [cam], poses, margin=1.5)
    out = R.render(prob, gt, poses)
    ups = tuple(torch.tensor(a.reshape(-1).astype(np.float32), device="cuda") for a in up)
    b = R.backward(gt, upstream=ups)
    counts = R.sync()
    return {k: v.cpu().numpy() for k, v in out.items()}, b, counts


@pytest.fixture(scope="module")
def default_run(case):
    g, cam, pose, gcfg, ref, up, ob = case
    R = gs.Rasterizer(gcfg)
    res = _run(R, g, cam, pose, up)
    R.close()
    return res


@pytest.mark.parametrize("sched", SCHEDULES)
def test_schedule_results_match_default_and_oracle(case, default_run, sched):
    g, cam, pose, gcfg, ref, up, ob = case
    base, b0, c0 = default_run
    R = gs.Rasterizer(gcfg)
    R.set_schedule(*sched)
    assert R.schedule == dict(zip(NAMES, sched + (0,)))
    out, b, counts = _run(R, g, cam, pose, up)
    R.close()
    assert counts.err_flags == 0 and counts.max_tile > max(sched[3], sched[4])
    if sched[:2] == (16, 16):
        assert counts.n_pairs == c0.n_pairs
    H, W = cam.height, cam.width
    _same_images(out, base, sched[:2] == (16, 16), ref["amb"], H, W)
    assert_images_close(out["rgb"].reshape(3, H, W), ref["rgb"], ref["amb"], what="rgb")
    assert_images_close(out["depth"].reshape(H, W), ref["depth"], ref["amb"], what="depth")
    assert_images_close(out["sil"].reshape(H, W), ref["sil"], ref["amb"], what="sil")
    for name, lo, hi in GRAD_KEYS:
        got = b["grads"][name].cpu().numpy().reshape(g.n, -1)
        assert_grads_close(got, ob["grads"][:, lo:hi], what=name)
        ri, r2 = rel_err(got, b0["grads"][name].cpu().numpy().reshape(g.n, -1))
        assert ri < 1e-5 and r2 < 1e-5, (name, ri, r2)
    assert_grads_close(b["pose_grad"].cpu().numpy()[0], ob["pose6"], what="pose")


def test_invalid_schedules_are_refused():
    R = gs.Rasterizer(gs.Config())
    for bad in [(16, 16, 3, 256, 256), (16, 16, 8, 256, 256), (16, 16, 4, 100, 256), (16, 16, 4, 256, 512),
                (16, 16, 4, 32, 256), (16, 16, 0, 64, 64), (8, 8, 4, 128, 64), (16, 8, 4, 128, 256),
                (4, 16, 4, 64, 64), (64, 4, 4, 64, 64), (8, 4, 4, 64, 64), (32, 16, 4, 256, 256),
                (12, 16, 4, 64, 64)]:
        with pytest.raises(gs.GsError):
            R.set_schedule(*bad)
    assert R.schedule == DEFAULT
    R.close()


def test_autotune_times_every_setting_and_keeps_results(case, default_run):
    g, cam, pose, gcfg, ref, up, ob = case
    base = default_run[0]
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    poses = torch.tensor(np.asarray(pose)[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [cam], poses, margin=3.0)  # room for the pairs of the smaller tiles
    tg = (torch.tensor(ref["rgb"].reshape(-1).astype(np.float32), device="cuda") * 0.9,
          torch.tensor(ref["depth"].reshape(-1).astype(np.float32), device="cuda") * 1.05, None)
    res = R.autotune(prob, gt, poses, tg, pose_only=False, reps=3)
    rows = res["timings_ms"]
    stages = [r["stage"] for r in rows]
    order = ("tile", "sub_buckets", "fwd_batch", "bwd_batch", "sort")  # no fused stage without pose_only
    assert stages == sorted(stages, key=order.index)
    # the tile shapes first, the context's own (the default) leading
    assert [(r["schedule"]["tile_w"], r["schedule"]["tile_h"]) for r in rows[:4]] == [(16, 16), (32, 8), (16, 8), (8, 8)]
    assert rows[0]["schedule"] == DEFAULT
    assert all(r["ms"] > 0 for r in rows)
    assert R.schedule == res["schedule"]
    for stage in order:
        cand = [r for r in rows if r["stage"] == stage]
        assert cand, stage
        timed = [r for r in cand if r["ms"] > 0]
        # each stage starts from the previous stage's choice and keeps it unless another
        # setting is at least 1 % faster
        first = cand[0]
        won = min(timed, key=lambda r: r["ms"])
        pick = won if won["ms"] < 0.99 * first["ms"] else first
        if stage == order[-1]:
            assert pick["schedule"] == res["schedule"]
        nxt = order + (None,)
        later = [r for r in rows if r["stage"] == nxt[nxt.index(stage) + 1]]
        if later:
            assert later[0]["schedule"] == pick["schedule"]
    # the tuned context renders the same images
    out, b, counts = _run(R, g, cam, pose, up)
    R.close()
    tile = (res["schedule"]["tile_w"], res["schedule"]["tile_h"])
    _same_images(out, base, tile == (16, 16), ref["amb"], cam.height, cam.width)


def test_tracking_graph_follows_the_schedule():
    """gs_track_step under a non-default schedule (the cached graph is keyed on it): the
    same pose as the default schedule to FP32 rounding after a few iterations."""
    g = scenes.room_scene(40_000, seed=4)
    cam = scenes.Cam(262.5, 262.5, 159.5, 119.5, 320, 240)
    truth = scenes.tracking_gt_pose()
    start = scenes.perturb_pose(truth, np.random.default_rng(5), 1.0, 0.03)
    rgb, depth = scenes.raycast_room(truth, cam, seed=4)
    frame = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rgb, depth)]
    gt = gs.GaussianTensors.from_numpy(g)
    s0 = torch.tensor(start, dtype=torch.float64, device="cuda")
    tr = slam.Tracker(cam, 5)
    out = []
    for sched in [(16, 16, 4, 256, 256), (16, 8, 1, 64, 128), (16, 16, 4, 256, 256), (16, 16, 4, 256, 256, 1),
                  (16, 8, 2, 128, 128, 1), (32, 8, 2, 64, 64, 1)]:
        tr.R.set_schedule(*sched)
        out.append(tr.track(gt, s0, *frame).cpu().numpy())
    tr.close()
    # the backward's atomics make even two runs of one schedule differ at rounding level
    assert np.abs(out[0] - out[2]).max() < 1e-6, np.abs(out[0] - out[2]).max()
    assert np.abs(out[0] - out[1]).max() < 1e-5, np.abs(out[0] - out[1]).max()
    # the fused compositing kernel (GS_SCHED_FUSED): the same arithmetic in one launch
    assert np.abs(out[0] - out[3]).max() < 1e-6, np.abs(out[0] - out[3]).max()
    for k in (4, 5):
        assert np.abs(out[0] - out[k]).max() < 1e-5, (k, np.abs(out[0] - out[k]).max())


def test_fused_tracking_kernel_matches_the_two_kernels():
    """One gs_track_step iteration with the forward and pose-only backward as two kernels
    and as k_track_tile (GS_SCHED_FUSED), for every batch depth: the loss to FP32
    summation order and the pose gradient (the first Adam moments over 1 - beta1) to 1e-5."""
    g = scenes.room_scene(40_000, seed=8)
    cam = scenes.Cam(262.5, 262.5, 159.5, 119.5, 320, 240)
    truth = scenes.tracking_gt_pose()
    start = scenes.perturb_pose(truth, np.random.default_rng(9), 1.0, 0.03)
    rgb, depth = scenes.raycast_room(truth, cam, seed=8)
    prior = scenes.prior_from_depth(depth, np.random.default_rng(3), 0.02, 0.05)
    tt = [torch.tensor(np.ascontiguousarray(a).reshape(-1), device="cuda") for a in (rgb, depth, prior)]
    tg = gs.gs_targets(*(x.data_ptr() for x in tt))
    gt = gs.GaussianTensors.from_numpy(g)
    for nb in (256, 128, 64):
        res = []
        for flags in (0, gs.GS_SCHED_FUSED):
            R = gs.Rasterizer(gs.Config())
            R.set_schedule(16, 16, 2, nb, nb, flags)
            poses = torch.tensor(np.asarray(start)[None], dtype=torch.float64, device="cuda")
            prob = R.plan(gt, [cam], poses, margin=1.5)
            ws, nbytes = R.workspace(prob)
            adam = torch.zeros(1, 16, dtype=torch.float64, device="cuda")
            hist = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
            gs.gs_track_step(R.ctx, prob, gt.c(), tg, poses, adam, hist, 1, ws, nbytes)
            R.sync()
            st = adam.cpu().numpy()[0]
            res.append((hist.item(), np.concatenate([st[0:3], st[6:9]]) / 0.1))
            R.close()
        (l0, g0), (l1, g1) = res
        assert l1 == pytest.approx(l0, rel=1e-6)
        assert np.abs(g1 - g0).max() <= 1e-5 * np.abs(g0).max(), (nb, g0, g1)


def test_tracker_tunes_on_the_first_frame_and_when_the_map_doubles():
    """slam.Tracker with autotune_reps: one gs_autotune on the first frame, none while the
    map keeps its size, another once it has doubled; the tracked pose matches an untuned
    tracker's to rounding (the tuned schedule may move the tile origins)."""
    g = scenes.room_scene(30_000, seed=6)
    cam = scenes.Cam(262.5, 262.5, 159.5, 119.5, 320, 240)
    truth = scenes.tracking_gt_pose()
    start = scenes.perturb_pose(truth, np.random.default_rng(7), 1.0, 0.03)
    rgb, depth = scenes.raycast_room(truth, cam, seed=6)
    frame = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rgb, depth)]
    gt = gs.GaussianTensors.from_numpy(g)
    s0 = torch.tensor(start, dtype=torch.float64, device="cuda")
    plain = slam.Tracker(cam, 5)
    p_plain = plain.track(gt, s0, *frame).cpu().numpy()
    plain.close()
    tr = slam.Tracker(cam, 5, autotune_reps=2)
    p1 = tr.track(gt, s0, *frame).cpu().numpy()
    assert tr.tunes == 1 and tr.tune["schedule"] == tr.R.schedule
    assert len(tr.tune["timings_ms"]) >= 7 and all(r["ms"] > 0 for r in tr.tune["timings_ms"])
    tr.track(gt, s0, *frame)
    assert tr.tunes == 1
    doubled = scenes.Gaussians(*(None if a is None else np.concatenate([a, a]) for a in g.arrays()))
    tr.track(gs.GaussianTensors.from_numpy(doubled), s0, *frame)
    assert tr.tunes == 1  # exactly twice the size: not more than double
    tripled = scenes.Gaussians(*(np.concatenate([a, a, a]) for a in g.arrays()))
    tr.track(gs.GaussianTensors.from_numpy(tripled), s0, *frame)
    assert tr.tunes == 2
    tr.close()
    assert np.abs(p1 - p_plain).max() < 1e-4, np.abs(p1 - p_plain).max()


def _sort_cases():
    """Scenes for the two sorts: the parity cube; a map listed twice (every depth tied
    with its copy, so the order of equal keys decides); a tile with 6,000 Gaussians (the
    per-tile sort's global-memory path); three views of uneven resolution (tile ids past
    eight bits, so the radix sort takes its second tile pass)."""
    g, cam = scenes.cube_scene(n=3000, seed=12)
    yield "cube", g, [cam], [scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(1), 1.0, 0.02)]
    d = scenes.Gaussians(*(np.concatenate([a, a]) for a in g.arrays()))
    yield "doubled", d, [cam], [scenes.identity_pose()]
    rng = np.random.default_rng(2)
    n = 6000
    means = np.stack([rng.normal(0, 0.01, n), rng.normal(0, 0.01, n), rng.uniform(1.0, 3.0, n)], 1)
    big = scenes.Gaussians(means.astype(np.float32), rng.normal(size=(n, 4)).astype(np.float32),
                           rng.normal(-4.5, 0.2, (n, 3)).astype(np.float32),
                           rng.normal(-3.0, 0.5, n).astype(np.float32), rng.uniform(size=(n, 3)).astype(np.float32))
    yield "long tile", big, [scenes.Cam(60.0, 60.0, 23.5, 23.5, 48, 48)], [scenes.identity_pose()]
    cams = [scenes.Cam(140.0, 140.0, 79.5, 59.5, 160, 120), scenes.Cam(70.0, 72.0, 39.5, 29.5, 80, 60),
            scenes.Cam(300.0, 300.0, 250.0, 150.0, 500, 300)]
    poses = [scenes.perturb_pose(scenes.identity_pose(), rng, 3.0, 0.05) for _ in cams]
    yield "three views", g, cams, poses


@pytest.mark.parametrize("case", list(_sort_cases()), ids=lambda c: c[0])
def test_radix_sort_gives_the_per_tile_order(case):
    """GS_SCHED_RADIX (one device-wide LSD radix sort of the (tile, depth) keys, ties put
    in Gaussian order afterwards) against the per-tile sort: the same front-to-back order,
    so bit-identical images, the same pair counts, and gradients equal to FP32 summation
    order; images against the oracle on its unambiguous pixels."""
    name, g, cams, poses = case
    gcfg, op = params_pair()
    runs = []
    for flags in (0, gs.GS_SCHED_RADIX):
        R = gs.Rasterizer(gcfg)
        R.set_schedule(16, 16, 4, 256, 256, flags)
        gt = gs.GaussianTensors.from_numpy(g)
        pz = torch.tensor(np.asarray(poses, dtype=np.float64).reshape(-1, 7), device="cuda")
        prob = R.plan(gt, cams, pz, margin=1.5)
        out = R.render(prob, gt, pz)
        P = sum(c.width * c.height for c in cams)
        rng = np.random.default_rng(7)
        ups = tuple(torch.tensor(rng.normal(size=k * P).astype(np.float32), device="cuda") for k in (3, 1, 1))
        b = R.backward(gt, upstream=ups, n_views=len(cams))
        counts = R.sync()
        assert counts.err_flags == 0
        runs.append(({k: v.cpu().numpy() for k, v in out.items()}, b, counts.n_pairs))
        R.close()
    (o0, b0, n0), (o1, b1, n1) = runs
    assert n0 == n1 > 0
    for k in ("rgb", "depth", "sil"):
        np.testing.assert_array_equal(o1[k], o0[k], err_msg=f"{name}: {k}")
    for gname in ("means", "quats", "log_scales", "logits", "rgb"):
        ri, r2 = rel_err(b1["grads"][gname].cpu().numpy(), b0["grads"][gname].cpu().numpy())
        assert ri < 1e-5 and r2 < 1e-5, (name, gname, ri, r2)
    ri, r2 = rel_err(b1["pose_grad"].cpu().numpy(), b0["pose_grad"].cpu().numpy())
    assert ri < 1e-5 and r2 < 1e-5, (name, "pose", ri, r2)
    off = 0
    for cam, pose in zip(cams, poses):
        H, W = cam.height, cam.width
        ref = oracle.render(oracle.Scene(*g.arrays()), ocam(cam), pose, op)
        rgb = o1["rgb"][3 * off:3 * (off + H * W)].reshape(3, H, W)
        assert_images_close(rgb, ref["rgb"], ref["amb"], what=f"{name} rgb")
        assert_images_close(o1["depth"][off:off + H * W].reshape(H, W), ref["depth"], ref["amb"], what=f"{name} depth")
        off += H * W


def test_radix_sort_in_the_tracking_graph():
    """gs_track_step with the radix sort, alone and with the fused compositor: the pose
    after three iterations equals the per-tile sort's to rounding."""
    g = scenes.room_scene(40_000, seed=4)
    cam = scenes.Cam(262.5, 262.5, 159.5, 119.5, 320, 240)
    truth = scenes.tracking_gt_pose()
    start = scenes.perturb_pose(truth, np.random.default_rng(5), 1.0, 0.03)
    rgb, depth = scenes.raycast_room(truth, cam, seed=4)
    frame = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (rgb, depth)]
    gt = gs.GaussianTensors.from_numpy(g)
    s0 = torch.tensor(start, dtype=torch.float64, device="cuda")
    tr = slam.Tracker(cam, 3)
    out = []
    for flags in (0, gs.GS_SCHED_RADIX, gs.GS_SCHED_RADIX | gs.GS_SCHED_FUSED):
        tr.R.set_schedule(16, 16, 4, 256, 256, flags)
        out.append(tr.track(gt, s0, *frame).cpu().numpy())
    tr.close()
    for k in (1, 2):
        assert np.abs(out[0] - out[k]).max() < 1e-6, (k, np.abs(out[0] - out[k]).max())
