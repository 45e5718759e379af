"""Pins of the map-side oracle (oracle/mapping.py) against what the paper and the
mathematics fix: the C oracle's own projection and compositing, closed forms of Adam,
and the invariants of a stable compaction."""
import numpy as np
import pytest

import oracle
from oracle import mapping as om
from paper_2408_05635_gb300 import scenes


def _frame(rng, cam, hole_frac=0.2):
    H, W = cam.height, cam.width
    depth = rng.uniform(0.5, 4.0, (H, W))
    depth[rng.uniform(size=(H, W)) < hole_frac] = 0.0
    return rng.uniform(size=(3, H, W)), depth


def _scene(new, rows=None):
    sel = slice(None) if rows is None else rows
    return oracle.Scene(new["means"][sel], new["quats"][sel], new["log_scales"][sel], new["logits"][sel].reshape(-1),
                        new["rgb"][sel])


def test_new_gaussians_project_onto_their_pixels():
    """Sec. III-A: the centre is the unprojected pixel and the radius depth / f makes the
    footprint one pixel wide: through the C oracle's pi_m every new Gaussian lands on
    its pixel (u, v) at depth d, and an isotropic s = d / f at depth d projects to
    Sigma' = I + t t^T px^2 with t = ((u - cx) / fx, (v - cy) / fy) the pixel's tangent
    (minor axis exactly one pixel; on the optical axis Sigma' = I)."""
    rng = np.random.default_rng(3)
    cam = oracle.camera(150.0, 150.0, 31.5, 23.5, 64, 48)
    rgb, depth = _frame(rng, cam)
    pose = scenes.perturb_pose(scenes.identity_pose(), rng, 20.0, 0.3)
    new = om.gaussians_from_frame(cam, pose, rgb, depth)
    assert new["pixel"].size == int((depth > 0).sum())
    pr = oracle.project(_scene(new), cam, pose, oracle.Params())
    v, u = np.divmod(new["pixel"], cam.width)
    np.testing.assert_allclose(pr["mu"][:, 0], u, atol=1e-9)
    np.testing.assert_allclose(pr["mu"][:, 1], v, atol=1e-9)
    np.testing.assert_allclose(pr["z"], depth.ravel()[new["pixel"]], rtol=1e-12)
    tx, ty = (u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy
    np.testing.assert_allclose(pr["cov2"], np.stack([1 + tx * tx, tx * ty, 1 + ty * ty], 1), atol=1e-9)
    np.testing.assert_array_equal(new["rgb"], rgb.reshape(3, -1)[:, new["pixel"]].T)


def test_new_gaussian_peak_is_half_opaque():
    """Rendered alone, a new Gaussian gives its pixel S = o = 0.5, C = 0.5 rgb, D = 0.5 d
    (Eqs. 2-4 at the peak of Eq. 1)."""
    rng = np.random.default_rng(4)
    cam = oracle.camera(120.0, 120.0, 15.5, 11.5, 32, 24)
    rgb, depth = _frame(rng, cam, hole_frac=0.0)
    pose = scenes.perturb_pose(scenes.identity_pose(), rng, 5.0, 0.1)
    new = om.gaussians_from_frame(cam, pose, rgb, depth)
    for k in (0, 137, 500):
        r = oracle.render(_scene(new, slice(k, k + 1)), cam, pose, oracle.Params())
        v, u = divmod(int(new["pixel"][k]), cam.width)
        assert r["sil"][v, u] == pytest.approx(0.5, abs=1e-12)
        assert r["depth"][v, u] == pytest.approx(0.5 * depth[v, u], rel=1e-12)
        np.testing.assert_allclose(r["rgb"][:, v, u], 0.5 * rgb[:, v, u], rtol=1e-12)


def test_keyframe_adds_only_unexplained_pixels():
    """Only pixels with depth and S < sil_add get a Gaussian, in row-major order."""
    rng = np.random.default_rng(5)
    cam = oracle.camera(100.0, 100.0, 19.5, 14.5, 40, 30)
    rgb, depth = _frame(rng, cam)
    sil = rng.uniform(size=depth.shape)
    new = om.gaussians_from_frame(cam, scenes.identity_pose(), rgb, depth, sil, sil_add=0.5)
    expect = np.flatnonzero(((depth > 0) & (sil < 0.5)).ravel())
    np.testing.assert_array_equal(new["pixel"], expect)
    assert np.all(np.diff(new["pixel"]) > 0)


# ---------------------------------------------------------------------------- Adam

def _groups(rng, n, scale=1.0):
    return {k: scale * rng.normal(size=(n, om.WIDTH[k])) for k in om.GROUPS}


LRS = {"means": 1e-4, "quats": 1e-3, "log_scales": 1e-3, "logits": 5e-2, "rgb": 2.5e-3}


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g from a zero state the bias-corrected moments are exactly
    m_hat = g and v_hat = g^2, so every step moves a parameter by lr g / (|g| + eps)."""
    rng = np.random.default_rng(6)
    p0, g = _groups(rng, 7), _groups(rng, 7, 1e-3)
    zero = {k: np.zeros_like(a) for k, a in p0.items()}
    p, m, v = p0, zero, zero
    eps = 1e-8
    for t in range(1, 6):
        p, m, v = om.adam_step(p, g, m, v, t, LRS, 0.9, 0.999, eps)
        for k in om.GROUPS:
            np.testing.assert_allclose(p[k], p0[k] - t * LRS[k] * g[k] / (np.abs(g[k]) + eps), rtol=0, atol=1e-12)


def test_adam_groups_use_their_own_rate():
    rng = np.random.default_rng(7)
    p0 = _groups(rng, 3)
    zero = {k: np.zeros_like(a) for k, a in p0.items()}
    g = {k: np.ones_like(a) for k, a in p0.items()}
    p, _, _ = om.adam_step(p0, g, zero, zero, 1, LRS, 0.9, 0.999, 0.0)
    for k in om.GROUPS:
        np.testing.assert_allclose(p0[k] - p[k], LRS[k], rtol=1e-12)


def test_adam_converges_on_a_quadratic():
    """Minimising sum (p - c)^2 drives every parameter to c."""
    rng = np.random.default_rng(8)
    c = _groups(rng, 5)
    p = _groups(rng, 5)
    m = {k: np.zeros_like(a) for k, a in p.items()}
    v = {k: np.zeros_like(a) for k, a in p.items()}
    lrs = {k: 0.05 for k in om.GROUPS}
    for t in range(1, 3001):
        g = {k: 2 * (p[k] - c[k]) for k in om.GROUPS}
        p, m, v = om.adam_step(p, g, m, v, t, lrs, 0.9, 0.999, 1e-12)
    for k in om.GROUPS:
        np.testing.assert_allclose(p[k], c[k], atol=2e-3)


# ---------------------------------------------------------------------------- removal

def test_prune_keeps_order_and_threshold():
    rng = np.random.default_rng(9)
    n = 1000
    logits = rng.normal(-4.0, 2.0, n).astype(np.float32)
    rows = np.arange(n)
    out = om.prune({"row": rows, "logit": logits}, logits, o_min=0.005)
    o = 1.0 / (1.0 + np.exp(-logits.astype(np.float64)))
    removed = np.setdiff1d(rows, out["row"])
    assert np.all(np.diff(out["row"]) > 0)
    assert np.all(o[out["row"]] >= 0.005 * (1 - 1e-6)) and np.all(o[removed] < 0.005 * (1 + 1e-6))
    assert 0 < out["row"].size < n
    np.testing.assert_array_equal(out["logit"], logits[out["row"]])


# ---------------------------------------------------------------------------- evaluation

def test_image_sums_and_psnr_closed_forms():
    from oracle import metrics as omx
    rng = np.random.default_rng(10)
    H, W = 12, 17
    rgb_t = rng.uniform(size=(3, H, W))
    depth_t = rng.uniform(0.5, 3.0, (H, W))
    depth_t[rng.uniform(size=(H, W)) < 0.3] = 0.0
    s = omx.image_sums(rgb_t + 0.1, depth_t + 0.02, rgb_t, depth_t)
    valid = int((depth_t > 0).sum())
    np.testing.assert_allclose(s, [3 * H * W * 0.01, 0.02 * valid, valid, 0.0004 * valid], rtol=1e-12)
    assert omx.psnr(s[0], 3 * H * W) == pytest.approx(20.0, abs=1e-9)
    assert omx.psnr(0.0, 10) == float("inf")


def test_trajectory_errors_closed_forms():
    from oracle import metrics as omx
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(11)
    gt = [scenes.perturb_pose(scenes.identity_pose(), rng, 30.0, 1.0) for _ in range(5)]
    e = omx.trajectory_errors(gt, gt)
    assert e["ate_rmse"] == 0.0 and np.allclose(e["rot"], 0.0, atol=1e-7)
    # moving every camera centre by a: world->camera t' = t - R a
    a = np.array([0.03, -0.04, 0.0])
    shifted = []
    for p in gt:
        R, t = scenes.pose_rt(p)
        shifted.append(scenes.pose_from_rt(R, t - R @ a))
    assert omx.trajectory_errors(shifted, gt)["ate_rmse"] == pytest.approx(0.05, rel=1e-9)
    # turning every camera by 0.1 rad about its own centre
    turned = []
    for p in gt:
        R, t = scenes.pose_rt(p)
        Q = Rotation.from_rotvec(0.1 * np.array([0.6, 0.0, 0.8])).as_matrix()
        turned.append(scenes.pose_from_rt(Q @ R, Q @ t))
    e = omx.trajectory_errors(turned, gt)
    np.testing.assert_allclose(e["rot"], 0.1, rtol=1e-9)
    assert e["ate_rmse"] == pytest.approx(0.0, abs=1e-12)


def test_ms_ssim_identities_and_closed_forms():
    """MS-SSIM of an image with itself is 1; of two constant images (no structure, so
    cs = 1 at every scale) it is l^b5 with l = (2 a b + C1) / (a^2 + b^2 + C1); it is
    symmetric, falls with added noise, and the window is the normalised Gaussian."""
    from oracle import metrics as omx
    rng = np.random.default_rng(12)
    img = rng.uniform(size=(3, 200, 260))
    assert omx.ms_ssim(img, img)["ms_ssim"] == pytest.approx(1.0, abs=1e-12)
    a, b = 0.3, 0.7
    c = omx.ms_ssim(np.full((3, 180, 180), a), np.full((3, 180, 180), b))
    lv = (2 * a * b + 1e-4) / (a * a + b * b + 1e-4)
    assert c["ms_ssim"] == pytest.approx(lv ** 0.1333, rel=1e-12)
    noisy = np.clip(img + rng.normal(0, 0.05, img.shape), 0, 1)
    noisier = np.clip(img + rng.normal(0, 0.2, img.shape), 0, 1)
    s1, s2 = omx.ms_ssim(img, noisy)["ms_ssim"], omx.ms_ssim(img, noisier)["ms_ssim"]
    assert 1.0 > s1 > s2 > 0.0
    assert omx.ms_ssim(noisy, img)["ms_ssim"] == pytest.approx(s1, rel=1e-12)
    g = omx.gaussian_window()
    assert g.sum() == pytest.approx(1.0) and np.argmax(g) == 5 and g[0] == pytest.approx(g[-1])
    # the 11-tap window samples a Gaussian of sigma 1.5: its second moment is sigma^2 less
    # the tails beyond +-5 px (0.3 %)
    x = np.arange(11) - 5.0
    assert float(np.sum(g * x * x)) == pytest.approx(1.5 ** 2, rel=5e-3)
    assert sum(omx.MSSSIM_WEIGHTS) == pytest.approx(1.0, abs=1e-3)


def test_ms_ssim_window_filter_is_a_valid_correlation():
    """The separable window filter equals scipy's 2-D correlation with the outer-product
    window over the valid positions."""
    from scipy.signal import correlate2d
    from oracle import metrics as omx
    rng = np.random.default_rng(13)
    img = rng.uniform(size=(37, 52))
    g = omx.gaussian_window()
    np.testing.assert_allclose(omx._filter_valid(img, g), correlate2d(img, np.outer(g, g), mode="valid"), rtol=1e-12)
