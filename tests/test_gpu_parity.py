"""GPU (CUDA path through the C ABI) vs the FP64 oracle on the same seeded inputs.

Images: max-abs <= 1e-4 on pixels the oracle marks unambiguous.  Gradients: per tensor
||gpu - oracle||_inf / ||oracle||_inf <= 1e-3 and the same in the 2-norm, with the same
upstream gradients (ambiguous pixels zeroed) fed to both backward passes.
"""
import numpy as np
import pytest
import torch

import oracle
import mask_model
from gpu_common import (assert_grads_close, assert_images_close, check_images, gpu_render, loss_tolerance, ocam,
                        params_pair, split_views)
from paper_2408_05635_gb300 import gs, scenes

pytestmark = pytest.mark.gpu

GRAD_KEYS = [("means", 0, 3), ("quats", 3, 7), ("log_scales", 7, 10), ("logits", 10, 11), ("rgb", 11, 14)]


def _scene_case(name):
    if name == "cube":
        g, cam = scenes.cube_scene()
        return g, cam
    if name == "ragged":
        g, _ = scenes.cube_scene(n=600, seed=3)
        return g, scenes.Cam(40.0, 44.0, 18.3, 11.1, 37, 23)
    raise KeyError(name)


@pytest.fixture(scope="module")
def cube():
    g, cam = scenes.cube_scene()
    rng = np.random.default_rng(0)
    target_pose = scenes.perturb_pose(scenes.identity_pose(), rng, 2.0, 0.03)
    return g, cam, target_pose, rng


@pytest.mark.parametrize("case", ["cube", "ragged"])
def test_forward_matches_oracle(case):
    g, cam = _scene_case(case)
    gcfg, op = params_pair()
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    pose = scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(5), 1.0, 0.02)
    out, prob, _, counts = gpu_render(R, gt, [cam], [pose])
    sc = oracle.Scene(*g.arrays())
    ref = oracle.render(sc, ocam(cam), pose, op)
    m = mask_model.mask_shares(sc, cam, pose, op, ref)
    assert m["alpha_min"] <= m["alpha_min_bound"] and m["t_min"] <= m["t_min_bound"], m
    check_images(out["rgb"], out["depth"], out["sil"], ref, sc, cam, pose, op, what=case)
    assert counts.n_pairs > 0 and counts.err_flags == 0


def test_fused_loss_matches_oracle(cube):
    g, cam, target_pose, rng = cube
    gcfg, op = params_pair()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    tgt = oracle.render(sc, oc, target_pose, op)
    prior = scenes.prior_from_depth(tgt["depth"], np.random.default_rng(1), 0.02, 0.05)
    t_rgb, t_depth = tgt["rgb"].astype(np.float32), tgt["depth"].astype(np.float32)
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    tt = tuple(torch.tensor(a.reshape(-1), device="cuda") for a in (t_rgb, t_depth, prior))
    out, prob, poses, _ = gpu_render(R, gt, [cam], [scenes.identity_pose()], targets=tt)
    ref = oracle.render(sc, oc, scenes.identity_pose(), op)
    L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], t_rgb, t_depth, prior)
    assert out["loss"][0] == pytest.approx(L["loss"], rel=2e-4)


def test_backward_matches_oracle(cube):
    """Same upstream gradients (the oracle's loss gradient, ambiguous pixels zeroed) into
    both backward passes; all 14 parameter gradients and the pose 6-vector compared."""
    g, cam, target_pose, rng = cube
    gcfg, op = params_pair()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    pose = scenes.identity_pose()
    tgt = oracle.render(sc, oc, target_pose, op)
    prior = scenes.prior_from_depth(tgt["depth"], np.random.default_rng(1), 0.02, 0.05)
    ref = oracle.render(sc, oc, pose, op)
    L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], tgt["rgb"], tgt["depth"], prior)
    mask = ref["amb"] | L["amb"]
    up_rgb = np.where(mask[None], 0.0, L["d_rgb"])
    up_d = np.where(mask, 0.0, L["d_depth"])
    up_s = np.where(mask, 0.0, L["d_sil"])
    ob = oracle.backward(sc, oc, pose, op, up_rgb, up_d, up_s)

    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    out, prob, poses, _ = gpu_render(R, gt, [cam], [pose])
    ups = tuple(torch.tensor(a.reshape(-1).astype(np.float32), device="cuda") for a in (up_rgb, up_d, up_s))
    b = R.backward(gt, upstream=ups)
    R.sync()
    for name, lo, hi in GRAD_KEYS:
        got = b["grads"][name].cpu().numpy().reshape(g.n, -1)
        assert_grads_close(got, ob["grads"][:, lo:hi], what=name)
    assert_grads_close(b["pose_grad"].cpu().numpy()[0], ob["pose6"], what="pose")


def test_pose_gradient_from_fused_loss(cube):
    """Pose gradient through the fused loss (no shared upstream): only a flagged pixel
    whose upstream gradient takes the other sign on one side can differ; the 6-vector
    agrees to the gradient bound 1e-3 (measured 7.5e-7)."""
    g, cam, target_pose, rng = cube
    gcfg, op = params_pair()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    tgt = oracle.render(sc, oc, target_pose, op)
    t_rgb, t_depth = tgt["rgb"].astype(np.float32), tgt["depth"].astype(np.float32)
    ref = oracle.render(sc, oc, scenes.identity_pose(), op)
    L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], t_rgb, t_depth, None)
    ob = oracle.backward(sc, oc, scenes.identity_pose(), op, L["d_rgb"], L["d_depth"], L["d_sil"])
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    tt = (torch.tensor(t_rgb.reshape(-1), device="cuda"), torch.tensor(t_depth.reshape(-1), device="cuda"), None)
    gpu_render(R, gt, [cam], [scenes.identity_pose()], targets=tt)
    b = R.backward(gt, params=False)
    R.sync()
    assert_grads_close(b["pose_grad"].cpu().numpy()[0], ob["pose6"], what="pose gradient through the fused loss")


def test_multi_view_uneven_resolution():
    g, _ = scenes.cube_scene(n=1500, seed=9)
    cams = [scenes.Cam(140.0, 140.0, 79.5, 59.5, 160, 120), scenes.Cam(70.0, 72.0, 39.5, 29.5, 80, 60),
            scenes.Cam(200.0, 200.0, 101.0, 48.0, 203, 97)]
    rng = np.random.default_rng(4)
    poses = [scenes.perturb_pose(scenes.identity_pose(), rng, 3.0, 0.05) for _ in cams]
    gcfg, op = params_pair()
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    out, prob, _, _ = gpu_render(R, gt, cams, poses)
    rgbs = split_views(out["rgb"], cams, 3)
    deps = split_views(out["depth"], cams, 1)
    sils = split_views(out["sil"], cams, 1)
    sc = oracle.Scene(*g.arrays())
    for k, (cam, pose) in enumerate(zip(cams, poses)):
        ref = oracle.render(sc, ocam(cam), pose, op)
        check_images(rgbs[k], deps[k], sils[k], ref, sc, cam, pose, op, what=f"view {k}")


def test_multi_block_scan_matches_single_view_calls():
    """40 views of 320 x 240 with 8 x 8 tiles and four sub-buckets per tile (192 k tile
    counters) take the multi-block scan; each view alone (4,800 counters) the one-block
    scan.  The images of the joint call equal those of the single-view calls bit for bit
    (the compositors sort each tile's list, so only the offsets and the launch order come
    from the scan), and the pair and record counts of the joint call are the sums of the
    single-view counts (the longest list their maximum)."""
    g, _ = scenes.cube_scene(n=3000, seed=11)
    cam = scenes.Cam(280.0, 280.0, 159.5, 119.5, 320, 240)
    rng = np.random.default_rng(12)
    poses = [scenes.perturb_pose(scenes.identity_pose(), rng, 4.0, 0.06) for _ in range(40)]
    gcfg, _ = params_pair()
    R = gs.Rasterizer(gcfg)
    R.set_schedule(8, 8, 4, 64, 64, 0)
    gt = gs.GaussianTensors.from_numpy(g)
    out, _, _, counts = gpu_render(R, gt, [cam] * 40, poses)
    assert 40 * (320 // 8) * (240 // 8) * 4 > 4 * 8192  # the multi-block form is taken
    n_pairs = n_records = 0
    max_tile = 0
    joint = {key: split_views(out[key], [cam] * 40, ch) for key, ch in (("rgb", 3), ("depth", 1), ("sil", 1))}
    for v, pose in enumerate(poses):
        one, _, _, c = gpu_render(R, gt, [cam], [pose])
        for key, ch in (("rgb", 3), ("depth", 1), ("sil", 1)):
            np.testing.assert_array_equal(joint[key][v].reshape(-1), one[key].reshape(-1), err_msg=f"view {v} {key}")
        n_pairs += int(c.n_pairs)
        n_records += int(c.n_records)
        max_tile = max(max_tile, int(c.max_tile))
    assert int(counts.n_pairs) == n_pairs
    assert int(counts.n_records) == n_records
    assert int(counts.max_tile) == max_tile


def test_long_tile_list_uses_global_sort():
    """More than 4096 Gaussians on one tile: the in-place global-memory sort path."""
    rng = np.random.default_rng(2)
    n = 6000
    means = np.stack([rng.normal(0, 0.01, n), rng.normal(0, 0.01, n), rng.uniform(1.0, 3.0, n)], 1)
    g = scenes.Gaussians(means.astype(np.float32), rng.normal(size=(n, 4)).astype(np.float32),
                         rng.normal(-4.5, 0.2, (n, 3)).astype(np.float32),
                         rng.normal(-3.0, 0.5, n).astype(np.float32), rng.uniform(size=(n, 3)).astype(np.float32))
    cam = scenes.Cam(60.0, 60.0, 23.5, 23.5, 48, 48)
    gcfg, op = params_pair()
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    out, prob, _, counts = gpu_render(R, gt, [cam], [scenes.identity_pose()])
    ref = oracle.render(oracle.Scene(*g.arrays()), ocam(cam), scenes.identity_pose(), op)
    assert_images_close(out["sil"].reshape(48, 48), ref["sil"], ref["amb"], what="sil")
    assert_images_close(out["depth"].reshape(48, 48), ref["depth"], ref["amb"], what="depth")


def test_large_footprints_listed_and_unlisted():
    """Key emission of large tile rectangles (more than 24 candidate tiles): 3,000 Gaussians
    a metre in front of a 160 x 120 camera, most covering about 6 x 6 of its 16 x 16 tiles,
    so every cell is crowded with them and the bounded list for k_emit's extra blocks
    (2,048 records) overflows: the listed records are emitted by those blocks, the rest by
    their cells' warps, and k_project counts both kinds block-wide.  Images against the
    oracle, and no capacity flag."""
    rng = np.random.default_rng(17)
    n = 3000
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.45, 0.45, n), rng.uniform(1.0, 1.6, n)], 1)
    g = scenes.Gaussians(means.astype(np.float32), rng.normal(size=(n, 4)).astype(np.float32),
                         rng.normal(-1.9, 0.15, (n, 3)).astype(np.float32),
                         rng.normal(-1.0, 0.5, n).astype(np.float32), rng.uniform(size=(n, 3)).astype(np.float32))
    cam = scenes.Cam(140.0, 140.0, 79.5, 59.5, 160, 120)
    gcfg, op = params_pair()
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    out, prob, _, counts = gpu_render(R, gt, [cam], [scenes.identity_pose()], margin=2.0)
    assert counts.err_flags == 0
    pr = oracle.project(oracle.Scene(*g.arrays()), ocam(cam), scenes.identity_pose(), op)
    b = pr["box"][pr["valid"]]  # pixel boxes, clipped to the image
    tiles = (b[:, 1] // 16 - b[:, 0] // 16 + 1) * (b[:, 3] // 16 - b[:, 2] // 16 + 1)
    assert (tiles > 24).sum() > 2048, (tiles > 24).sum()
    sc = oracle.Scene(*g.arrays())
    ref = oracle.render(sc, ocam(cam), scenes.identity_pose(), op)
    check_images(out["rgb"], out["depth"], out["sil"], ref, sc, cam, scenes.identity_pose(), op,
                 what="large footprints")


def test_empty_and_culled_scenes():
    gcfg, op = params_pair()
    R = gs.Rasterizer(gcfg)
    cam = scenes.Cam(50.0, 50.0, 15.5, 11.5, 32, 24)
    # every Gaussian behind the camera
    g, _ = scenes.cube_scene(n=300, seed=1)
    g.means[:, 2] *= -1
    out, _, _, counts = gpu_render(R, gs.GaussianTensors.from_numpy(g), [cam], [scenes.identity_pose()])
    assert counts.n_records == 0 and counts.n_pairs == 0
    assert np.all(out["rgb"] == 0) and np.all(out["sil"] == 0) and np.all(out["depth"] == 0)


def test_capacity_overflow_is_reported_not_fatal():
    g, cam = scenes.cube_scene()
    R = gs.Rasterizer(gs.Config())
    gt = gs.GaussianTensors.from_numpy(g)
    poses = torch.tensor(scenes.identity_pose()[None], dtype=torch.float64, device="cuda")
    prob = R.problem(g.n, [cam], pair_capacity=100)
    R.render(prob, gt, poses)
    st, c = gs.gs_sync_status(R.ctx)
    assert st == gs.GS_ERR_CAPACITY
    assert c.err_flags & gs.ERR_PAIRS and c.n_pairs > 100
    # the flags are cleared and the context stays usable
    prob = R.plan(gt, [cam], poses)
    R.render(prob, gt, poses)
    assert R.sync().err_flags == 0


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_low_precision_attributes(dtype):
    """BF16 / FP16 attributes (means stay FP32): same bounds against the oracle run on the
    dequantized attributes; the error against the FP32-attribute oracle is reported."""
    g, cam = scenes.cube_scene()
    gq = scenes.Gaussians(g.means, *(torch.tensor(a).to(dtype).float().numpy() for a in
                                     (g.quats, g.log_scales, g.logits, g.rgb)))
    gcfg, op = params_pair()
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g, attr_dtype=dtype)
    out, _, _, _ = gpu_render(R, gt, [cam], [scenes.identity_pose()])
    ref = oracle.render(oracle.Scene(*gq.arrays()), ocam(cam), scenes.identity_pose(), op)
    H, W = cam.height, cam.width
    assert_images_close(out["rgb"].reshape(3, H, W), ref["rgb"], ref["amb"], what="rgb")
    assert_images_close(out["depth"].reshape(H, W), ref["depth"], ref["amb"], what="depth")


def _track_setup(g, cam, t_rgb, t_depth, prior, start, margin=2.0):
    R = gs.Rasterizer(gs.Config())
    gt = gs.GaussianTensors.from_numpy(g)
    poses = torch.tensor(np.asarray(start)[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [cam], poses, margin=margin)
    ws, nb = R.workspace(prob)
    keep = [torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float32, device="cuda")
            for a in (t_rgb, t_depth) + ((prior,) if prior is not None else ())]
    targets = gs.gs_targets(keep[0].data_ptr(), keep[1].data_ptr(), keep[2].data_ptr() if prior is not None else None)
    adam = torch.zeros(1, 16, dtype=torch.float64, device="cuda")
    return R, gt, poses, prob, ws, nb, targets, adam, keep


def _pose_diff(a, b):
    from scipy.spatial.transform import Rotation
    Ra, ta = scenes.pose_rt(a)
    Rb, tb = scenes.pose_rt(b)
    return (float(np.linalg.norm(-Ra.T @ ta + Rb.T @ tb)),
            float(np.linalg.norm(Rotation.from_matrix(Ra @ Rb.T).as_rotvec())))


def test_track_step_follows_oracle(cube):
    """Decoupled tracking on the GPU (CUDA graph, fused loss, FP64 Adam on the device):
    the first update equals the oracle's Adam step on the oracle's gradient, and ten
    iterations stay on the oracle's trajectory (Adam moves each coordinate by at most
    lr per step, so one sign flip of a near-zero gradient component costs 2 lr)."""
    g, cam, target_pose, rng = cube
    op = oracle.Params()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    tgt = oracle.render(sc, oc, target_pose, op)
    t_rgb, t_depth = tgt["rgb"].astype(np.float32), tgt["depth"].astype(np.float32)
    start = scenes.identity_pose()
    R, gt, poses, prob, ws, nb, targets, adam, keep = _track_setup(g, cam, t_rgb, t_depth, None, start)
    hist = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
    gs.gs_track_step(R.ctx, prob, gt.c(), targets, poses, adam, hist, 1, ws, nb)
    R.sync()
    ref = oracle.render(sc, oc, start, op)
    L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], t_rgb, t_depth, None)
    ob = oracle.backward(sc, oc, start, op, L["d_rgb"], L["d_depth"], L["d_sil"])
    o_pose, o_state = oracle.adam_step(start, np.zeros(16), ob["pose6"], op)
    np.testing.assert_allclose(poses.cpu().numpy()[0], o_pose, atol=1e-9)
    tol = loss_tolerance(L["loss"], ref, sc, cam, start, op, t_rgb, t_depth, None)
    assert abs(hist.item() - L["loss"]) <= tol, (hist.item(), L["loss"], tol)
    hist = torch.zeros(9, 1, dtype=torch.float64, device="cuda")
    gs.gs_track_step(R.ctx, prob, gt.c(), targets, poses, adam, hist, 9, ws, nb)
    R.sync()
    pose = o_pose
    losses = []
    for _ in range(9):
        r = oracle.render(sc, oc, pose, op)
        L = oracle.loss(oc, op, r["rgb"], r["depth"], r["sil"], t_rgb, t_depth, None)
        losses.append(L["loss"])
        b = oracle.backward(sc, oc, pose, op, L["d_rgb"], L["d_depth"], L["d_sil"])
        pose, o_state = oracle.adam_step(pose, o_state, b["pose6"], op)
    dc, dr = _pose_diff(poses.cpu().numpy()[0], pose)
    print(f"10-iteration trajectory gap: centre {dc:.2e} m, rotation {dr:.2e} rad")
    np.testing.assert_allclose(hist.cpu().numpy()[:, 0], losses, rtol=5e-3)
    assert dc < 4 * op.lr_trans and dr < 4 * op.lr_rot


def test_track_step_converges_on_room():
    """Sanity (not parity): 40 GPU tracking iterations on the 320 x 240 room from a start
    2 deg / 5 cm away move the camera toward the ground truth."""
    g = scenes.room_scene(200_000, seed=0)
    cam = scenes.QVGA_CAM
    gtp = scenes.tracking_gt_pose()
    rng = np.random.default_rng(1)
    start = scenes.perturb_pose(gtp, rng, 2.0, 0.05)
    rgb, depth = scenes.raycast_room(gtp, cam)
    prior = scenes.prior_from_depth(depth, rng, 0.02, 0.05)
    R, gt, poses, prob, ws, nb, targets, adam, keep = _track_setup(g, cam, rgb, depth, prior, start)
    hist = torch.zeros(40, 1, dtype=torch.float64, device="cuda")
    gs.gs_track_step(R.ctx, prob, gt.c(), targets, poses, adam, hist, 40, ws, nb)
    R.sync()
    c0, r0 = _pose_diff(start, gtp)
    c1, r1 = _pose_diff(poses.cpu().numpy()[0], gtp)
    print(f"room tracking: centre {c0:.3f} -> {c1:.3f} m, rotation {np.degrees(r0):.2f} -> {np.degrees(r1):.2f} deg")
    assert c1 < 0.8 * c0 and r1 < 0.5 * r0


def test_mapping_window_grads_sum_over_views():
    """Mapping (Sec. III-C): parameter gradients of the combined loss summed over a
    window of keyframes, processed a chunk of views at a time (lists recomputed per
    chunk).  Against the oracle's per-view gradients of the same loss, summed, to the
    gradient bound 1e-3 (the fused loss differentiates every pixel, flagged ones too, whose
    upstream sign may differ; measured 3e-5), each view's loss to what its flagged pixels'
    FP32 outcomes allow (loss_tolerance); and chunk sizes 1 and 4 agree to float-atomic
    order."""
    g = scenes.room_scene(60_000, seed=3)
    cam = scenes.Cam(150.0, 150.0, 79.5, 44.5, 160, 90)
    poses_np = scenes.mapping_keyframes(4)
    gcfg, op = params_pair()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    rng = np.random.default_rng(5)
    targets, ref_grads, ref_loss, loss_tol = [], np.zeros((g.n, 14)), [], []
    for pose in poses_np:
        t = oracle.render(sc, oc, scenes.perturb_pose(pose, rng, 0.5, 0.01), op)
        prior = scenes.prior_from_depth(t["depth"], rng, 0.03, 0.08)
        t_rgb, t_depth = t["rgb"].astype(np.float32), t["depth"].astype(np.float32)
        r = oracle.render(sc, oc, pose, op)
        L = oracle.loss(oc, op, r["rgb"], r["depth"], r["sil"], t_rgb, t_depth, prior)
        ref_grads += oracle.backward(sc, oc, pose, op, L["d_rgb"], L["d_depth"], L["d_sil"])["grads"]
        ref_loss.append(L["loss"])
        loss_tol.append(loss_tolerance(L["loss"], r, sc, cam, pose, op, t_rgb, t_depth, prior))
        targets.append(tuple(torch.tensor(a.reshape(-1), device="cuda") for a in (t_rgb, t_depth, prior)))
    gt = gs.GaussianTensors.from_numpy(g)
    poses = torch.tensor(np.stack(poses_np), dtype=torch.float64, device="cuda")
    outs = {}
    for chunk in (1, 2, 4):
        R = gs.Rasterizer(gcfg)
        outs[chunk] = R.mapping_grads(gt, [cam] * 4, poses, targets, chunk=chunk)
        R.sync()
    assert np.all(np.abs(outs[2]["loss"].cpu().numpy() - np.asarray(ref_loss)) <= np.asarray(loss_tol)), loss_tol
    for name, lo, hi in GRAD_KEYS:
        got = outs[2]["grads"][name].cpu().numpy().reshape(g.n, -1)
        assert_grads_close(got, ref_grads[:, lo:hi], what=name)
        a = outs[1]["grads"][name].cpu().numpy()
        b = outs[4]["grads"][name].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-5 * max(1e-30, np.abs(a).max()), name


def _opaque_stacks(n_stacks=24, layers=4, seed=21):
    """Stacks of nearly opaque Gaussians in front of the cube scene: each stack puts
    `layers` Gaussians 5 cm apart in depth over nearly the same pixels, opacities from
    sigmoid(6) = 0.9975 (clamped at alpha_max = 0.99) down to sigmoid(3) = 0.95, so the
    reverse walk recovers the transmittance through factors 1 / (1 - alpha) of up to 100."""
    g, _ = scenes.cube_scene(n=600, seed=seed)
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-0.45, 0.45, size=(n_stacks, 2))
    means, logits = [], []
    for s in range(n_stacks):
        for k in range(layers):
            means.append([xy[s, 0] + rng.normal(0, 0.004), xy[s, 1] + rng.normal(0, 0.004), 1.2 + 0.05 * k])
            logits.append([6.0, 4.0, 5.0, 3.0][k % 4])
    m = len(means)
    stack = scenes.Gaussians(np.asarray(means, np.float32), rng.normal(size=(m, 4)).astype(np.float32),
                             rng.normal(-3.2, 0.15, size=(m, 3)).astype(np.float32), np.asarray(logits, np.float32),
                             rng.uniform(0, 1, size=(m, 3)).astype(np.float32))
    cat = lambda a, b: np.concatenate([a, b])
    return scenes.Gaussians(*(cat(a, b) for a, b in zip(stack.arrays(), g.arrays())))


@pytest.mark.parametrize("t_min", [1e-4, 1e-6])
def test_backward_through_near_opaque_stacks(t_min):
    """Images and all gradients where the transmittance is rebuilt by division through
    stacks of alpha = 0.95 .. 0.99 Gaussians (relative error up to 100 u per layer), with
    the default early stop and with t_min = 1e-6, which lets three clamped layers through."""
    g = _opaque_stacks()
    cam = scenes.Cam(100.0, 100.0, 47.5, 35.5, 96, 72)
    pose = scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(8), 0.5, 0.01)
    gcfg, op = params_pair(t_min=t_min)
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    ref = oracle.render(sc, oc, pose, op)
    # the stacks really are opaque: many pixels end below 1e-3 transmittance
    assert (ref["sil"] > 1 - 1e-3).mean() > 0.05
    R = gs.Rasterizer(gcfg)
    gt = gs.GaussianTensors.from_numpy(g)
    out, prob, poses, _ = gpu_render(R, gt, [cam], [pose])
    H, W = cam.height, cam.width
    amb = ref["amb"]
    assert_images_close(out["rgb"].reshape(3, H, W), ref["rgb"], amb, what="rgb")
    assert_images_close(out["depth"].reshape(H, W), ref["depth"], amb, what="depth")
    rng = np.random.default_rng(5)
    up = [np.where(amb[None], 0.0, rng.normal(size=(3, H, W))), np.where(amb, 0.0, rng.normal(size=(H, W))),
          np.where(amb, 0.0, rng.normal(size=(H, W)))]
    ob = oracle.backward(sc, oc, pose, op, *up)
    ups = tuple(torch.tensor(a.reshape(-1).astype(np.float32), device="cuda") for a in up)
    b = R.backward(gt, upstream=ups)
    R.sync()
    for name, lo, hi in GRAD_KEYS:
        got = b["grads"][name].cpu().numpy().reshape(g.n, -1)
        assert_grads_close(got, ob["grads"][:, lo:hi], what=name)
    assert_grads_close(b["pose_grad"].cpu().numpy()[0], ob["pose6"], what="pose")
