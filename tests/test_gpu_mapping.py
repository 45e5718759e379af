"""Scene-optimisation kernels (gs_map_add, gs_map_adam_step, gs_map_prune) against the
map-side oracle, through the C ABI.

Index and copy work (which pixels become Gaussians and in what order, which Gaussians
survive removal, moved moments and low-precision copies) must match bit for bit;
floating-point results within the rounding of the FP32 arithmetic: unprojected means to
1e-6 m, log-scales to 1e-6, Adam moments and parameters within bounds carried through
the recursion (the first moment's rounding is relative to the sum of |terms|).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import assert_images_close, ocam
from oracle import mapping as om
from paper_2408_05635_gb300 import gs, scenes

pytestmark = pytest.mark.gpu

CAM = scenes.Cam(140.0, 150.0, 79.5, 59.5, 160, 120)


def _lrs(cfg):
    return {"means": cfg.lr_means, "quats": cfg.lr_quats, "log_scales": cfg.lr_log_scales,
            "logits": cfg.lr_opacity_logits, "rgb": cfg.lr_rgb}


def _groups(iso):
    return ("means", "log_scales", "logits", "rgb") if iso else om.GROUPS


def _width(iso):
    return dict(om.WIDTH, log_scales=1) if iso else om.WIDTH


def _state_views(state, cap, iso=False):
    """Split the flat Adam state into per-group (m, v) arrays of capacity rows."""
    off, out = 0, {}
    per = sum(_width(iso)[k] for k in _groups(iso))
    for k in _groups(iso):
        w = _width(iso)[k]
        out[k] = (state[off * cap:(off + w) * cap].reshape(cap, w),
                  state[(per + off) * cap:(per + off + w) * cap].reshape(cap, w))
        off += w
    return out


def _frame(pose, cam=CAM, seed=0):
    rgb, depth = scenes.raycast_room(pose, cam, seed=seed)
    return np.ascontiguousarray(rgb, np.float32), np.ascontiguousarray(depth, np.float32)


# ---------------------------------------------------------------------------- Adam

@pytest.mark.parametrize("lowp,iso", [(None, False), (torch.bfloat16, False), (torch.float16, True)])
def test_adam_steps_match_oracle(lowp, iso):
    rng = np.random.default_rng(1)
    n, cap = 1001, 1004
    M = gs.Map(cap, lowp_dtype=lowp, isotropic=iso)
    cap = M.capacity
    G, Wd = _groups(iso), _width(iso)
    p0 = {k: rng.normal(size=(cap, Wd[k])).astype(np.float32) for k in G}
    for k in G:
        M.p[k].copy_(torch.from_numpy(p0[k].reshape(M.p[k].shape)))
        if M.lp is not None and k != "means":
            M.lp[k].copy_(M.p[k].to(lowp))
    M.count.fill_(n)
    cfg = M.config
    p = {k: p0[k][:n].astype(np.float64) for k in G}
    m = {k: np.zeros_like(a) for k, a in p.items()}
    v = {k: np.zeros_like(a) for k, a in p.items()}
    # error bounds of the FP32 recursion (u = 2^-24): m sums terms of either sign, so its
    # rounding is relative to m_abs, the same recursion on |g|; the step's ratio carries
    # that error divided by sqrt(v_hat) plus a few roundings of its own
    u = 2.0 ** -24
    m_abs = {k: np.zeros_like(a) for k, a in p.items()}
    p_err = {k: np.zeros_like(a) for k, a in p.items()}
    for t in range(1, 4):
        g = {k: (rng.normal(size=(cap, Wd[k])) * 10.0 ** rng.uniform(-4, 1, (cap, 1))).astype(np.float32)
             for k in G}
        gt = {k: torch.from_numpy(g[k].reshape(M.p[k].shape)).cuda() for k in G}
        if t == 3:
            gt.pop("rgb")  # a group without a gradient is left alone
        M.adam_step(gt, t)
        gg = {k: g[k][:n].astype(np.float64) for k in G}
        q, m2, v2 = om.adam_step(p, gg, m, v, t, _lrs(cfg), cfg.beta1, cfg.beta2, cfg.eps, groups=G)
        for k in G:
            if t == 3 and k == "rgb":
                continue
            m_abs[k] = cfg.beta1 * m_abs[k] + (1 - cfg.beta1) * np.abs(gg[k])
            c1, c2 = 1 / (1 - cfg.beta1 ** t), 1 / (1 - cfg.beta2 ** t)
            den = np.sqrt(v2[k] * c2) + cfg.eps
            ratio = m2[k] * c1 / den
            p_err[k] += 2 * u * np.abs(q[k]) + _lrs(cfg)[k] * (8 * u * m_abs[k] * c1 / den + 6 * u * np.abs(ratio))
        if t == 3:
            q["rgb"], m2["rgb"], v2["rgb"] = p["rgb"], m["rgb"], v["rgb"]
        p, m, v = q, m2, v2
    torch.cuda.synchronize()
    st = _state_views(M.state.cpu().numpy(), cap, iso)
    for k in G:
        got = M.p[k].cpu().numpy().reshape(cap, -1)
        lr = _lrs(cfg)[k]
        assert np.all(np.abs(got[:n] - p[k]) <= p_err[k] + 1e-7 * lr), k
        np.testing.assert_array_equal(got[n:], p0[k][n:], err_msg=f"{k} rows past n")
        assert np.all(np.abs(st[k][0][:n] - m[k]) <= 8 * u * m_abs[k] + 1e-30), f"{k} m"
        np.testing.assert_allclose(st[k][1][:n], v[k], rtol=4 * 6 * u, atol=1e-30, err_msg=f"{k} v")
        assert not st[k][0][n:].any() and not st[k][1][n:].any()
        if lowp is not None and k != "means":
            np.testing.assert_array_equal(M.lp[k].float().cpu().numpy(), M.p[k].to(lowp).float().cpu().numpy())


# ---------------------------------------------------------------------------- new Gaussians

def _check_added(M, n0, ref, state_before=None):
    n1 = M.n
    k = ref["pixel"].size
    assert n1 == n0 + k
    iso = M.isotropic
    got = {key: M.p[key][n0:n1].cpu().numpy().reshape(k, -1).astype(np.float64) for key in M.GROUPS}
    np.testing.assert_array_equal(got["rgb"], ref["rgb"].astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(got["means"], ref["means"], rtol=0, atol=1e-6)
    np.testing.assert_allclose(got["log_scales"], ref["log_scales"][:, :1] if iso else ref["log_scales"], rtol=0,
                               atol=1e-6)
    if not iso:
        np.testing.assert_array_equal(got["quats"], ref["quats"])
    np.testing.assert_array_equal(got["logits"], ref["logits"])
    if M.state is not None:
        st = _state_views(M.state.cpu().numpy(), M.capacity, iso)
        for key in M.GROUPS:
            assert not st[key][0][n0:n1].any() and not st[key][1][n0:n1].any()
            if state_before is not None:
                sb = _state_views(state_before, M.capacity, iso)
                np.testing.assert_array_equal(st[key][0][:n0], sb[key][0][:n0])
    if M.lp is not None:
        for key in M.GROUPS[1:]:
            np.testing.assert_array_equal(M.lp[key][n0:n1].float().cpu().numpy(),
                                          M.p[key][n0:n1].to(M.lowp_dtype).float().cpu().numpy())


@pytest.mark.parametrize("iso", [False, True])
def test_first_frame_gaussians_match_oracle(iso):
    """Sec. III-A: one Gaussian per pixel with depth, in pixel order, at the start of an
    empty map (anisotropic, or isotropic as Eq. 1 is written)."""
    pose = scenes.look_at((2.5, 1.5, 0.8), (0.2, -0.1, 1.0))
    rgb, depth = _frame(pose)
    M = gs.Map(CAM.width * CAM.height, lowp_dtype=torch.float16, isotropic=iso)
    M.add_from_frame(CAM, torch.tensor(pose, dtype=torch.float64, device="cuda"), torch.from_numpy(rgb).cuda(),
                     torch.from_numpy(depth).cuda())
    ref = om.gaussians_from_frame(ocam(CAM), pose, rgb, depth)
    assert 0 < ref["pixel"].size
    _check_added(M, 0, ref)
    assert M.err.item() == 0


def test_keyframe_adds_where_silhouette_is_low():
    """Sec. III-C: on a keyframe only pixels with S < sil_add; appended after the live
    Gaussians, whose parameters and moments stay as they were."""
    rng = np.random.default_rng(2)
    pose = scenes.look_at((1.5, 1.2, 1.5), (1.0, 0.1, 0.4))
    rgb, depth = _frame(pose)
    sil = rng.uniform(size=depth.shape).astype(np.float32)
    M = gs.Map(40000)
    n0 = 37
    for k in om.GROUPS:
        M.p[k].normal_()
    M.state.normal_()
    M.count.fill_(n0)
    before = M.state.cpu().numpy()
    M.add_from_frame(CAM, torch.tensor(pose, dtype=torch.float64, device="cuda"), torch.from_numpy(rgb).cuda(),
                     torch.from_numpy(depth).cuda(), torch.from_numpy(sil).cuda())
    ref = om.gaussians_from_frame(ocam(CAM), pose, rgb, depth, sil, sil_add=M.config.sil_add)
    _check_added(M, n0, ref, before)


def test_add_overflow_fills_to_capacity_and_flags():
    pose = scenes.look_at((2.5, 1.5, 0.8), (0.0, 0.0, 1.0))
    rgb, depth = _frame(pose)
    M = gs.Map(1000)
    M.add_from_frame(CAM, torch.tensor(pose, dtype=torch.float64, device="cuda"), torch.from_numpy(rgb).cuda(),
                     torch.from_numpy(depth).cuda())
    assert M.n == M.capacity and M.err.item() & 1
    ref = om.gaussians_from_frame(ocam(CAM), pose, rgb, depth)
    got = M.p["rgb"].cpu().numpy()
    np.testing.assert_array_equal(got, ref["rgb"][:M.capacity].astype(np.float32))


# ---------------------------------------------------------------------------- removal

@pytest.mark.parametrize("n,iso", [(0, False), (1, False), (5000, False), (5000, True)])
def test_prune_matches_oracle(n, iso):
    rng = np.random.default_rng(3)
    cap = 5004
    A = gs.Map(cap, lowp_dtype=torch.bfloat16, isotropic=iso)
    B = gs.Map(cap, lowp_dtype=torch.bfloat16, isotropic=iso)
    for k in A.GROUPS:
        A.p[k].normal_()
    A.p["logits"].copy_(torch.from_numpy(rng.normal(-5.3, 0.6, cap).astype(np.float32)))
    for k in A.GROUPS[1:]:
        A.lp[k].copy_(A.p[k].to(torch.bfloat16))
    A.state.normal_()
    A.count.fill_(n)
    B.count.fill_(12345)
    A.prune_into(B)
    logits = A.p["logits"].cpu().numpy()[:n]
    keep = om.keep_mask(logits, A.config.opacity_min)
    k = int(keep.sum())
    assert B.n == k
    if n == 5000:
        assert 0 < k < n
    for key in A.GROUPS:
        np.testing.assert_array_equal(B.p[key][:k].cpu().numpy(), A.p[key][:n].cpu().numpy()[keep])
        if key != "means":
            np.testing.assert_array_equal(B.lp[key][:k].float().cpu().numpy(), A.lp[key][:n].float().cpu().numpy()[keep])
    sa, sb = _state_views(A.state.cpu().numpy(), A.capacity, iso), _state_views(B.state.cpu().numpy(), B.capacity, iso)
    for key in A.GROUPS:
        np.testing.assert_array_equal(sb[key][0][:k], sa[key][0][:n][keep])
        np.testing.assert_array_equal(sb[key][1][:k], sa[key][1][:n][keep])


# ---------------------------------------------------------------------------- end to end

def test_first_frame_map_renders_like_the_oracle():
    """The first-frame map rendered from its own pose: GPU (gs_map_add + gs_project +
    gs_forward) against the oracle rendering the oracle's own first-frame Gaussians."""
    pose = scenes.look_at((2.5, 1.5, 0.8), (0.2, -0.1, 1.0))
    rgb, depth = _frame(pose)
    M = gs.Map(CAM.width * CAM.height)
    pt = torch.tensor(np.asarray(pose)[None], dtype=torch.float64, device="cuda")
    M.add_from_frame(CAM, pt[0], torch.from_numpy(rgb).cuda(), torch.from_numpy(depth).cuda())
    R = gs.Rasterizer(gs.Config())
    g = M.gaussians()
    prob = R.plan(g, [CAM], pt, margin=1.5)
    out = R.render(prob, g, pt)
    R.sync()
    ref_g = om.gaussians_from_frame(ocam(CAM), pose, rgb, depth)
    # the oracle renders what the GPU stores: its FP32 rounding of the oracle's Gaussians
    f32 = {k: ref_g[k].astype(np.float32).astype(np.float64) for k in om.GROUPS}
    sc = oracle.Scene(f32["means"], f32["quats"], f32["log_scales"], f32["logits"].reshape(-1), f32["rgb"])
    ref = oracle.render(sc, ocam(CAM), pose, oracle.Params())
    H, W = CAM.height, CAM.width
    assert ref["amb"].mean() < 0.05
    assert_images_close(out["rgb"].cpu().numpy().reshape(3, H, W), ref["rgb"], ref["amb"], what="rgb")
    assert_images_close(out["depth"].cpu().numpy().reshape(H, W), ref["depth"], ref["amb"], what="depth")
    assert_images_close(out["sil"].cpu().numpy().reshape(H, W), ref["sil"], ref["amb"], what="sil")
    # every pixel with depth is covered at least by its own half-opaque Gaussian
    assert np.all(ref["sil"][depth > 0] >= 0.5 - 1e-9)


def test_mapping_iterations_reduce_the_loss():
    """Sec. III-C end to end on the GPU: a map initialised from one keyframe, made opaque
    (so every pixel with depth is inside the loss mask S > 0.99 from the start and the
    mask does not grow under the optimisation) and its colours scrambled, optimised
    against two keyframes (poses fixed) with gs_map_adam_step: the window loss falls."""
    poses = [scenes.look_at((2.5, 1.5, 0.8), (0.0, 0.0, 1.0)), scenes.look_at((2.4, 1.5, 0.9), (0.1, 0.0, 1.0))]
    frames = [_frame(p) for p in poses]
    M = gs.Map(CAM.width * CAM.height)
    pt = torch.tensor(np.asarray(poses), dtype=torch.float64, device="cuda")
    M.add_from_frame(CAM, pt[0], torch.from_numpy(frames[0][0]).cuda(), torch.from_numpy(frames[0][1]).cuda())
    n = M.n
    M.p["rgb"][:n] = torch.rand(n, 3, device="cuda")
    M.p["logits"][:n] = 5.0
    R = gs.Rasterizer(gs.Config())
    targets = [(torch.from_numpy(f[0]).cuda(), torch.from_numpy(f[1]).cuda(), None) for f in frames]
    losses = []
    grads = {k: torch.zeros_like(M.p[k]) for k in om.GROUPS}
    for it in range(1, 41):
        for t in grads.values():
            t.zero_()
        g = M.gaussians(n)
        out = R.mapping_grads(g, [CAM, CAM], pt, targets, chunk=2,
                              grads={"means": grads["means"][:n], "quats": grads["quats"][:n],
                                     "log_scales": grads["log_scales"][:n], "logits": grads["logits"][:n],
                                     "rgb": grads["rgb"][:n]})
        losses.append(float(out["loss"].sum()))
        M.adam_step(grads, it)
    R.sync()
    assert losses[-1] < 0.85 * losses[0], losses
    # (Adam's first step moves every parameter by its full rate and may raise it briefly)
    assert losses[-1] < min(losses[:10]), losses
