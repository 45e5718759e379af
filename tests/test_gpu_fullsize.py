"""Full-size parity: the workloads and launch configurations that bench.py times,
checked against the FP64 oracle on what it can compute at that size.

* Tracking frame (640 x 480, 200k room Gaussians, FP32): the whole frame's images, the
  loss, all parameter gradients and the pose gradient at the start pose, and the first
  graph-launched tracking update (gs_track_step).
* Batched hypotheses (32 keyframes of uneven resolution x 16 pose hypotheses, 500k room
  Gaussians, BF16 attributes, one call for all 512 views): one sampled view per
  resolution, against the oracle run on the dequantized attributes: images, per-view
  loss, pose gradient (upstream given on the sampled views only, so every other view's
  pose gradient must be exactly zero), and the first graph-launched update.
* Mapping window (8 keyframes 1200 x 680, 1M room Gaussians, FP32): one keyframe's
  images, its 14 parameter gradients and its pose gradient.

The batched views include Gaussians within a few cm of the near plane (cameras right
above the room's boxes): their thin screen covariances are inverted with a cancellation-
free determinant (k_project), and the Jacobian of those whose mean lies far outside the
view is taken at the clamped image-plane tangent.  The oracle masks the pixels whose
discrete decisions an FP32 renderer may take differently (gs_oracle.c); the fraction is
printed and bounded.

Tolerances as in the small parity tests: images 1e-4 max-abs on unambiguous pixels,
gradients 1e-3 relative (inf and 2-norm) with the ambiguous pixels' upstream zeroed on
both sides; losses and fused-loss updates include the ambiguous pixels and use the
stated looser bounds.
"""
import numpy as np
import pytest
import torch

import bench
import oracle
import mask_model
from gpu_common import assert_grads_close, assert_images_close, check_images, loss_tolerance, ocam
from paper_2408_05635_gb300 import gs, scenes

pytestmark = pytest.mark.gpu

GRAD_KEYS = [("means", 0, 3), ("quats", 3, 7), ("log_scales", 7, 10), ("logits", 10, 11), ("rgb", 11, 14)]


def _masked_upstream(ref, L):
    mask = ref["amb"] | L["amb"]
    return (np.where(mask[None], 0.0, L["d_rgb"]), np.where(mask, 0.0, L["d_depth"]),
            np.where(mask, 0.0, L["d_sil"]), mask)


# ---------------------------------------------------------------------------- tracking frame

@pytest.fixture(scope="module")
def tracking():
    g, cam, gt_pose, start, rgb, depth, prior = bench.workload()
    op = oracle.Params()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    ref = oracle.render(sc, oc, start, op)
    L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], rgb, depth, prior)
    targets = tuple(torch.tensor(a.reshape(-1), device="cuda") for a in (rgb, depth, prior))
    return dict(g=g, cam=cam, start=start, op=op, sc=sc, oc=oc, ref=ref, L=L, targets=targets,
                frame=(rgb, depth, prior))


def test_tracking_frame_images_and_loss(tracking):
    t = tracking
    R = gs.Rasterizer(gs.Config())
    gt = gs.GaussianTensors.from_numpy(t["g"])
    poses = torch.tensor(np.asarray(t["start"])[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [t["cam"]], poses, margin=1.5)
    out = R.render(prob, gt, poses, targets=t["targets"])
    R.sync()
    ref = t["ref"]
    # the flagged share is what the mask's margins predict (closed forms, mask_model)
    m = mask_model.mask_shares(t["sc"], t["cam"], t["start"], t["op"], ref)
    print(f"tracking frame mask: {m}")
    assert m["alpha_min"] <= m["alpha_min_bound"] and m["t_min"] <= m["t_min_bound"], m
    check_images(out["rgb"].cpu().numpy(), out["depth"].cpu().numpy(), out["sil"].cpu().numpy(), ref, t["sc"],
                 t["cam"], t["start"], t["op"], what="tracking frame")
    tol = loss_tolerance(t["L"]["loss"], ref, t["sc"], t["cam"], t["start"], t["op"], *t["frame"])
    assert abs(out["loss"].item() - t["L"]["loss"]) <= tol, (out["loss"].item(), t["L"]["loss"], tol)


def test_tracking_frame_gradients(tracking):
    t = tracking
    up_rgb, up_d, up_s, _ = _masked_upstream(t["ref"], t["L"])
    ob = oracle.backward(t["sc"], t["oc"], t["start"], t["op"], up_rgb, up_d, up_s)
    R = gs.Rasterizer(gs.Config())
    gt = gs.GaussianTensors.from_numpy(t["g"])
    poses = torch.tensor(np.asarray(t["start"])[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [t["cam"]], poses, margin=1.5)
    R.render(prob, gt, poses, images=False)
    ups = tuple(torch.tensor(a.reshape(-1).astype(np.float32), device="cuda") for a in (up_rgb, up_d, up_s))
    b = R.backward(gt, upstream=ups)
    R.sync()
    n = t["g"].n
    for name, lo, hi in GRAD_KEYS:
        assert_grads_close(b["grads"][name].cpu().numpy().reshape(n, -1), ob["grads"][:, lo:hi], what=name)
    assert_grads_close(b["pose_grad"].cpu().numpy()[0], ob["pose6"], what="pose")


@pytest.mark.parametrize("flags", [0, gs.GS_SCHED_FUSED])
def test_tracking_graph_first_update(tracking, flags):
    """The bench's launch: gs_track_step (CUDA graph) from the start pose, with the two
    compositing kernels and with the fused one (GS_SCHED_FUSED).  The first decoupled
    Adam step moves each coordinate by lr * g / (|g| + eps), which the fused loss's
    ambiguous pixels do not change unless a gradient component is near zero; the first
    moments it leaves are (1 - beta1) g, the pose gradient itself, which must match the
    oracle's through the same (unmasked) loss to the gradient bound 1e-3 (a flagged pixel
    can flip the sign of its upstream gradient on either side; measured 5e-6 here), and
    the loss to what the flagged pixels' FP32 outcomes allow (loss_tolerance)."""
    t = tracking
    L = t["L"]
    ob = oracle.backward(t["sc"], t["oc"], t["start"], t["op"], L["d_rgb"], L["d_depth"], L["d_sil"])
    o_pose, _ = oracle.adam_step(t["start"], np.zeros(16), ob["pose6"], t["op"])
    R = gs.Rasterizer(gs.Config())
    R.set_schedule(16, 16, 4, 256, 256, flags)
    gt = gs.GaussianTensors.from_numpy(t["g"])
    poses = torch.tensor(np.asarray(t["start"])[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [t["cam"]], poses, margin=1.5)
    ws, nb = R.workspace(prob)
    tg = gs.gs_targets(*(x.data_ptr() for x in t["targets"]))
    adam = torch.zeros(1, 16, dtype=torch.float64, device="cuda")
    hist = torch.zeros(1, 1, dtype=torch.float64, device="cuda")
    gs.gs_track_step(R.ctx, prob, gt.c(), tg, poses, adam, hist, 1, ws, nb)
    R.sync()
    np.testing.assert_allclose(poses.cpu().numpy()[0], o_pose, atol=1e-9)
    tol = loss_tolerance(L["loss"], t["ref"], t["sc"], t["cam"], t["start"], t["op"], *t["frame"])
    assert abs(hist.item() - L["loss"]) <= tol, (hist.item(), L["loss"], tol)
    st = adam.cpu().numpy()[0]
    g6 = np.concatenate([st[0:3], st[6:9]]) / (1.0 - t["op"].beta1)
    assert_grads_close(g6, ob["pose6"], what="pose gradient through the fused loss")


def test_tracking_with_host_upload_equals_device_targets(tracking):
    """gs_track_step_upload: the frame in page-locked host memory is either copied into the
    device targets beside the first iteration's binning, or (targets NULL) read in place by
    the kernels.  Five iterations from the start pose give, in both forms, the poses,
    losses and Adam state of gs_track_step on the device frame to the run-to-run spread of
    the FP32 gradient atomics, whose order is not fixed (poses 1e-7 absolute: Adam's step
    lr g / (|g| + eps) moves a coordinate with a near-zero gradient by that noise; losses
    1e-6 relative; moments 1e-4 relative); the device targets hold the host frame after the
    copy (they start as NaN); the host result holds the last pose and loss (stored there by
    the device); and a frame in ordinary (pageable) host memory is refused in both forms."""
    t = tracking
    R = gs.Rasterizer(gs.Config())
    R.set_schedule(16, 16, 4, 256, 256, gs.GS_SCHED_FUSED)
    gt = gs.GaussianTensors.from_numpy(t["g"])
    start = torch.tensor(np.asarray(t["start"])[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [t["cam"]], start, margin=1.5)
    ws, nb = R.workspace(prob)
    out = []
    for mode in ("device", "copy", "in_place"):
        poses = start.clone()
        adam = torch.zeros(1, 16, dtype=torch.float64, device="cuda")
        hist = torch.zeros(5, 1, dtype=torch.float64, device="cuda")
        if mode != "device":
            dev = tuple(torch.full_like(x, float("nan")) for x in t["targets"])
            host = tuple(x.cpu().pin_memory() for x in t["targets"])
            result = torch.full((8,), float("nan"), dtype=torch.float64).pin_memory()
            src = gs.gs_host_targets(*(x.data_ptr() for x in host), result.data_ptr())
            tg = gs.gs_targets(*(x.data_ptr() for x in dev)) if mode == "copy" else None
            gs.gs_track_step_upload(R.ctx, prob, gt.c(), tg, src, poses, adam, hist, 5, ws, nb)
        else:
            tg = gs.gs_targets(*(x.data_ptr() for x in t["targets"]))
            gs.gs_track_step(R.ctx, prob, gt.c(), tg, poses, adam, hist, 5, ws, nb)
        R.sync()
        out.append((poses.cpu().numpy(), hist.cpu().numpy(), adam.cpu().numpy()))
        if mode != "device":
            for d, h in zip(dev, host):
                if mode == "copy":
                    assert torch.equal(d.cpu(), h)
                else:  # read in place: the device buffers are not touched
                    assert torch.isnan(d).all()
            # the last iteration's pose and loss, stored into host memory by the device
            np.testing.assert_array_equal(result.numpy()[:7], out[-1][0][0])
            assert result.numpy()[7] == out[-1][1][-1, 0]
            pageable = tuple(x.cpu() for x in t["targets"])
            bad = gs.gs_host_targets(*(x.data_ptr() for x in pageable), None)
            with pytest.raises(gs.GsError):
                gs.gs_track_step_upload(R.ctx, prob, gt.c(), tg, bad, poses, adam, hist, 1, ws, nb)
    p0, h0, a0 = out[0]
    for p1, h1, a1 in out[1:]:
        np.testing.assert_allclose(p1, p0, rtol=0, atol=1e-7)
        np.testing.assert_allclose(h1, h0, rtol=1e-6)
        np.testing.assert_allclose(a1, a0, rtol=1e-4, atol=1e-9 * np.abs(a0).max())


# ---------------------------------------------------------------------------- batched hypotheses

@pytest.fixture(scope="module")
def batched():
    g, cams, poses0, frame_of, frames = bench.batched_workload()
    # the oracle runs on what the GPU reads: BF16-rounded attributes, FP32 means
    gq = scenes.Gaussians(g.means, *(torch.tensor(a).to(torch.bfloat16).float().numpy() for a in
                                     (g.quats, g.log_scales, g.logits, g.rgb)))
    sample = []
    for w in sorted({c.width for c in cams}):
        sample.append(next(v for v, c in enumerate(cams) if c.width == w))
    pix = np.array([c.width * c.height for c in cams])
    off = np.concatenate([[0], np.cumsum(pix)])
    op = oracle.Params()
    sc = oracle.Scene(*gq.arrays())
    refs = {}
    for v in sample:
        oc = ocam(cams[v])
        rgb, depth, prior = frames[frame_of[v]]
        ref = oracle.render(sc, oc, poses0[v], op)
        L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], rgb, depth, prior)
        refs[v] = (oc, ref, L, (rgb, depth, prior))
    t_rgb = torch.cat([torch.from_numpy(frames[f][0].reshape(-1)) for f in frame_of]).cuda()
    t_depth = torch.cat([torch.from_numpy(frames[f][1].reshape(-1)) for f in frame_of]).cuda()
    t_prior = torch.cat([torch.from_numpy(frames[f][2].reshape(-1)) for f in frame_of]).cuda()
    gt = gs.GaussianTensors.from_numpy(g, attr_dtype=torch.bfloat16)
    return dict(g=g, cams=cams, poses0=poses0, sample=sample, off=off, op=op, sc=sc, refs=refs, gt=gt,
                targets=(t_rgb, t_depth, t_prior))


def test_batched_sampled_views_images_and_loss(batched):
    b = batched
    R = gs.Rasterizer(gs.Config())
    poses = torch.tensor(np.asarray(b["poses0"]), dtype=torch.float64, device="cuda")
    prob = R.plan(b["gt"], b["cams"], poses, margin=1.5)
    out = R.render(prob, b["gt"], poses, targets=b["targets"])
    R.sync()
    off = b["off"]
    for v in b["sample"]:
        oc, ref, L, tg_v = b["refs"][v]
        H, W = oc.height, oc.width
        # the flagged share is what the mask's margins predict (closed forms, mask_model)
        m = mask_model.mask_shares(b["sc"], oc, b["poses0"][v], b["op"], ref)
        print(f"view {v} ({W}x{H}) mask: {m}")
        assert m["alpha_min"] <= m["alpha_min_bound"] and m["t_min"] <= m["t_min_bound"], m
        check_images(out["rgb"][3 * off[v]:3 * off[v + 1]].cpu().numpy(), out["depth"][off[v]:off[v + 1]].cpu().numpy(),
                     out["sil"][off[v]:off[v + 1]].cpu().numpy(), ref, b["sc"], oc, b["poses0"][v], b["op"],
                     what=f"batched view {v}")
        tol = loss_tolerance(L["loss"], ref, b["sc"], oc, b["poses0"][v], b["op"], *tg_v)
        assert abs(out["loss"][v].item() - L["loss"]) <= tol, (v, out["loss"][v].item(), L["loss"], tol)


def test_batched_sampled_views_pose_gradient(batched):
    b = batched
    off = b["off"]
    P = int(off[-1])
    up = torch.zeros(5 * P, dtype=torch.float32, device="cuda")
    ups = (up[:3 * P], up[3 * P:4 * P], up[4 * P:])
    expect = {}
    for v in b["sample"]:
        oc, ref, L, tg_v = b["refs"][v]
        u_rgb, u_d, u_s, _ = _masked_upstream(ref, L)
        ups[0][3 * off[v]:3 * off[v + 1]] = torch.tensor(u_rgb.reshape(-1).astype(np.float32), device="cuda")
        ups[1][off[v]:off[v + 1]] = torch.tensor(u_d.reshape(-1).astype(np.float32), device="cuda")
        ups[2][off[v]:off[v + 1]] = torch.tensor(u_s.reshape(-1).astype(np.float32), device="cuda")
        expect[v] = oracle.backward(b["sc"], oc, b["poses0"][v], b["op"], u_rgb, u_d, u_s)["pose6"]
    R = gs.Rasterizer(gs.Config())
    poses = torch.tensor(np.asarray(b["poses0"]), dtype=torch.float64, device="cuda")
    prob = R.plan(b["gt"], b["cams"], poses, margin=1.5)
    R.render(prob, b["gt"], poses, images=False)
    out = R.backward(b["gt"], upstream=ups, params=False, n_views=len(b["cams"]))
    R.sync()
    pg = out["pose_grad"].cpu().numpy()
    for v in b["sample"]:
        assert_grads_close(pg[v], expect[v], what=f"pose view {v}")
    others = np.setdiff1d(np.arange(len(b["cams"])), b["sample"])
    assert np.all(pg[others] == 0.0)


def test_batched_graph_first_update(batched):
    """The batched bench launch: one gs_track_step for all 512 views; the sampled views'
    first decoupled Adam step equals the oracle's on the oracle's fused-loss gradient."""
    b = batched
    V = len(b["cams"])
    R = gs.Rasterizer(gs.Config())
    poses = torch.tensor(np.asarray(b["poses0"]), dtype=torch.float64, device="cuda")
    prob = R.plan(b["gt"], b["cams"], poses, margin=1.5)
    ws, nb = R.workspace(prob)
    tg = gs.gs_targets(*(x.data_ptr() for x in b["targets"]))
    adam = torch.zeros(V, 16, dtype=torch.float64, device="cuda")
    hist = torch.zeros(1, V, dtype=torch.float64, device="cuda")
    gs.gs_track_step(R.ctx, prob, b["gt"].c(), tg, poses, adam, hist, 1, ws, nb)
    R.sync()
    got = poses.cpu().numpy()
    for v in b["sample"]:
        oc, ref, L, tg_v = b["refs"][v]
        ob = oracle.backward(b["sc"], oc, b["poses0"][v], b["op"], L["d_rgb"], L["d_depth"], L["d_sil"])
        o_pose, _ = oracle.adam_step(b["poses0"][v], np.zeros(16), ob["pose6"], b["op"])
        np.testing.assert_allclose(got[v], o_pose, atol=1e-9, err_msg=f"view {v}")
        tol = loss_tolerance(L["loss"], ref, b["sc"], oc, b["poses0"][v], b["op"], *tg_v)
        assert abs(hist[0, v].item() - L["loss"]) <= tol, (v, hist[0, v].item(), L["loss"], tol)


# ---------------------------------------------------------------------------- mapping window

def test_mapping_keyframe_gradients():
    """One keyframe of the mapping window (1200 x 680, 1M room Gaussians): its images, all
    14 parameter gradients and the pose gradient against the oracle, with the oracle's loss
    gradient (ambiguous pixels zeroed) as the shared upstream."""
    g, cams, poses_np, frames = bench.mapping_workload()
    v = 1
    cam, pose = cams[v], poses_np[v]
    rgb, depth, prior = frames[v]
    op = oracle.Params()
    sc, oc = oracle.Scene(*g.arrays()), ocam(cam)
    ref = oracle.render(sc, oc, pose, op)
    L = oracle.loss(oc, op, ref["rgb"], ref["depth"], ref["sil"], rgb, depth, prior)
    up_rgb, up_d, up_s, mask = _masked_upstream(ref, L)
    m = mask_model.mask_shares(sc, cam, pose, op, ref)
    print(f"mapping keyframe mask: {m}; with the loss mask's own decisions {mask.mean():.4%}")
    assert m["alpha_min"] <= m["alpha_min_bound"] and m["t_min"] <= m["t_min_bound"], m
    ob = oracle.backward(sc, oc, pose, op, up_rgb, up_d, up_s)
    R = gs.Rasterizer(gs.Config())
    gt = gs.GaussianTensors.from_numpy(g)
    poses = torch.tensor(np.asarray(pose)[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [cam], poses, margin=1.25)
    out = R.render(prob, gt, poses)
    check_images(out["rgb"].cpu().numpy(), out["depth"].cpu().numpy(), out["sil"].cpu().numpy(), ref, sc, cam, pose,
                 op, what="mapping keyframe")
    ups = tuple(torch.tensor(a.reshape(-1).astype(np.float32), device="cuda") for a in (up_rgb, up_d, up_s))
    b = R.backward(gt, upstream=ups)
    R.sync()
    for name, lo, hi in GRAD_KEYS:
        assert_grads_close(b["grads"][name].cpu().numpy().reshape(g.n, -1), ob["grads"][:, lo:hi], what=name)
    assert_grads_close(b["pose_grad"].cpu().numpy()[0], ob["pose6"], what="pose")
