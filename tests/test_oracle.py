"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a closed form,
an invariant, a brute-force or finite-difference computation, a Monte-Carlo estimate or
a hand-worked fixture under tests/golden/.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from conftest import oracle_cam, oracle_scene
from paper_2408_05635_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _single(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, rgb=(0.2, 0.6, 0.9)):
    return oracle.Scene(np.array([mean], float), np.array([quat], float),
                        np.full((1, 3), log_scale) if np.isscalar(log_scale) else np.array([log_scale], float),
                        np.array([logit], float), np.array([rgb], float))


def _smooth_params(**kw):
    """Thresholds off: every Gaussian contributes everywhere, the maps are smooth."""
    return oracle.Params(alpha_min=0.0, alpha_max=1.0, t_min=0.0, **kw)


# ----------------------------------------------------------------------------- projection

def test_single_gaussian_golden():
    """Eq. 1 / pi_m / Eqs. 2-4 for one isotropic Gaussian on the optical axis (hand-derived)."""
    gold = json.load(open(os.path.join(GOLDEN, "single_gaussian.json")))
    sc = _single((0, 0, 2.0), math.log(0.02))
    cam = oracle.camera(140, 140, 10, 8, 21, 17)
    p = oracle.Params()
    pr = oracle.project(sc, cam, scenes.identity_pose(), p)
    np.testing.assert_allclose(pr["cov2"][0], gold["cov2"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pr["mu"][0], gold["mu"], rtol=0, atol=1e-12)
    r = oracle.render(sc, cam, scenes.identity_pose(), p)
    pk = gold["peak"]
    assert r["sil"][8, 10] == pytest.approx(pk["sil"], abs=1e-14)
    np.testing.assert_allclose(r["rgb"][:, 8, 10], pk["rgb"], atol=1e-14)
    assert r["depth"][8, 10] == pytest.approx(pk["depth"], abs=1e-14)
    assert r["t_final"][8, 10] == pytest.approx(pk["t_final"], abs=1e-14)
    assert r["sil"][8, 11] == pytest.approx(gold["neighbour_11_8_sil"], rel=1e-12)
    # support: non-zero exactly inside the radius (pixel centres), zero outside
    yy, xx = np.mgrid[0:17, 0:21]
    rho = np.hypot(xx - 10, yy - 8)
    rad = gold["support_radius_px"]
    assert np.all(r["sil"][rho < rad - 1e-6] > 0)
    assert np.all(r["sil"][rho > rad + 1e-6] == 0)


def test_projection_pinhole_and_depth(rng):
    """pi_m (Sec. II-A) with the world->camera pose: mu' = (fx X/Z + cx, fy Y/Z + cy) with
    (X, Y, Z) = R x + t, the rotation taken from scipy rather than the oracle."""
    n = 50
    means = rng.uniform([-1, -1, 2], [1, 1, 4], size=(n, 3))
    sc = oracle.Scene(means, rng.normal(size=(n, 4)), np.full((n, 3), -4.0), np.zeros(n), np.full((n, 3), 0.5))
    pose = scenes.perturb_pose(scenes.identity_pose(), rng, 5.0, 0.1)
    R, t = scenes.pose_rt(pose)
    cam = oracle.camera(300, 310, 160.3, 118.7, 320, 240)
    pr = oracle.project(sc, cam, pose, oracle.Params())
    xc = means @ R.T + t
    np.testing.assert_allclose(pr["z"], xc[:, 2], rtol=1e-13)
    np.testing.assert_allclose(pr["mu"][:, 0], 300 * xc[:, 0] / xc[:, 2] + 160.3, rtol=1e-12)
    np.testing.assert_allclose(pr["mu"][:, 1], 310 * xc[:, 1] / xc[:, 2] + 118.7, rtol=1e-12)


def test_projection_covariance_monte_carlo():
    """Sigma' = J W Sigma W^T J^T: sample 3-D points from N(x, R s s^T R^T) (scipy
    rotation), push them through the pinhole and compare the empirical 2-D covariance."""
    rng = np.random.default_rng(7)
    q = np.array([0.3, -0.5, 0.7, 0.2])
    ls = np.log([0.004, 0.012, 0.002])
    mean = np.array([0.4, -0.3, 2.5])
    pose = scenes.perturb_pose(scenes.identity_pose(), rng, 20.0, 0.05)
    cam = oracle.camera(500, 480, 320, 240, 640, 480)
    sc = oracle.Scene(mean[None], q[None], ls[None], np.zeros(1), np.full((1, 3), 0.5))
    pr = oracle.project(sc, cam, pose, oracle.Params())
    Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    L = Rg @ np.diag(np.exp(ls))
    pts = mean + rng.normal(size=(400_000, 3)) @ L.T
    R, t = scenes.pose_rt(pose)
    xc = pts @ R.T + t
    uv = np.stack([500 * xc[:, 0] / xc[:, 2], 480 * xc[:, 1] / xc[:, 2]], 1)
    emp = np.cov(uv.T)
    A, B, C = pr["cov2"][0]
    np.testing.assert_allclose([A, B, C], [emp[0, 0], emp[0, 1], emp[1, 1]], rtol=1.5e-2, atol=2e-3 * A)
    # the conic is the inverse of Sigma'
    a, b, c = pr["conic"][0]
    np.testing.assert_allclose(np.array([[a, b], [b, c]]) @ np.array([[A, B], [B, C]]), np.eye(2), atol=1e-12)


def test_jacobian_clamp_beyond_view():
    """Beyond +-jac_clip half-extents the Jacobian is frozen: sliding a Gaussian sideways
    at a fixed depth moves its screen mean as pi_m says but leaves Sigma' unchanged, and
    Sigma' is continuous where the clamp begins; inside the clamp it equals the unclamped
    Sigma'."""
    cam = oracle.camera(200, 200, 160, 120, 320, 240)
    lim = 1.3 * 160 / 200  # tangent limit along x at the default jac_clip
    z = 1.0
    xs = np.array([0.5 * lim, lim * (1 - 1e-9), lim * (1 + 1e-9), 1.5 * lim, 4.0 * lim, 9.0 * lim])
    n = xs.size
    q = np.tile([0.9, 0.2, -0.3, 0.25], (n, 1))
    sc = oracle.Scene(np.stack([xs * z, np.full(n, 0.1), np.full(n, z)], 1), q, np.tile(np.log([0.01, 0.03, 0.2]), (n, 1)),
                      np.zeros(n), np.full((n, 3), 0.5))
    pr = oracle.project(sc, cam, scenes.identity_pose(), oracle.Params(alpha_min=0.0))
    free = oracle.project(sc, cam, scenes.identity_pose(), oracle.Params(alpha_min=0.0, jac_clip=0.0))
    np.testing.assert_allclose(pr["mu"][:, 0], 200 * xs + 160, rtol=1e-12)
    np.testing.assert_allclose(pr["cov2"][:2], free["cov2"][:2], rtol=1e-12)
    np.testing.assert_allclose(pr["cov2"][1], pr["cov2"][2], rtol=1e-7)
    for k in (3, 4, 5):
        np.testing.assert_allclose(pr["cov2"][k], pr["cov2"][2], rtol=1e-12)
    # unclamped, the footprint of the far mean is stretched many times over
    assert free["cov2"][5, 0] > 20 * pr["cov2"][5, 0]


def test_near_plane_culls():
    sc = oracle.Scene(np.array([[0, 0, 0.15], [0, 0, 1.0]]), np.tile([1.0, 0, 0, 0], (2, 1)),
                      np.full((2, 3), -3.0), np.zeros(2), np.full((2, 3), 0.5))
    pr = oracle.project(sc, oracle.camera(100, 100, 32, 24, 64, 48), scenes.identity_pose(), oracle.Params())
    assert list(pr["valid"]) == [False, True]


# ----------------------------------------------------------------------------- compositing

def test_two_gaussians_closed_form():
    """Eqs. 2-4 for two Gaussians under one pixel: S = 1 - (1-a1)(1-a2), C = c1 a1 +
    c2 a2 (1-a1), D = z1 a1 + z2 a2 (1-a1), whatever their index order."""
    cam = oracle.camera(100, 100, 5, 5, 11, 11)
    p = oracle.Params()
    # index 0 is the far one; the near one must still be composited first
    sc = oracle.Scene(np.array([[0, 0, 3.0], [0, 0, 2.0]]), np.tile([1.0, 0, 0, 0], (2, 1)),
                      np.full((2, 3), math.log(0.03)), np.array([0.4, -0.7]),
                      np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.5]]))
    r = oracle.render(sc, cam, scenes.identity_pose(), p)
    a_far, a_near = 1 / (1 + math.exp(-0.4)), 1 / (1 + math.exp(0.7))
    assert r["sil"][5, 5] == pytest.approx(1 - (1 - a_near) * (1 - a_far), abs=1e-14)
    np.testing.assert_allclose(r["rgb"][:, 5, 5], np.array([0, 1, 0.5]) * a_near + np.array([1, 0, 0]) * a_far * (1 - a_near),
                               atol=1e-14)
    assert r["depth"][5, 5] == pytest.approx(2.0 * a_near + 3.0 * a_far * (1 - a_near), abs=1e-14)
    assert r["n_contrib"][5, 5] == 2


def test_alpha_clamp_and_early_stop():
    """alpha is clamped at alpha_max, and the walk stops before the Gaussian that would
    drop the transmittance below t_min (reading of the paper's silent thresholds)."""
    cam = oracle.camera(100, 100, 5, 5, 11, 11)
    n = 4
    sc = oracle.Scene(np.array([[0, 0, 1.0 + k] for k in range(n)], float), np.tile([1.0, 0, 0, 0], (n, 1)),
                      np.full((n, 3), math.log(0.05)), np.full(n, 12.0), np.eye(3)[[0, 1, 2, 0]])
    p = oracle.Params(alpha_max=0.99, t_min=1e-4)
    r = oracle.render(sc, cam, scenes.identity_pose(), p)
    # alpha = 0.99 twice -> T = 1e-4, the third would take it to 1e-6 < t_min: stop there
    assert r["n_contrib"][5, 5] == 2
    assert r["t_final"][5, 5] == pytest.approx(0.01 * 0.01, rel=1e-12)
    np.testing.assert_allclose(r["rgb"][:, 5, 5], [0.99, 0.01 * 0.99, 0], atol=1e-14)


def test_compositing_invariants_cube():
    """On the 160 x 120 cube scene: S + T_final = 1, 0 <= S <= 1, T_final >= t_min,
    min z S <= D <= max z S, C_ch <= max c S (Eqs. 2-4 are convex-combination-like)."""
    g, cam = scenes.cube_scene()
    sc, oc = oracle_scene(g), oracle_cam(cam)
    p = oracle.Params()
    r = oracle.render(sc, oc, scenes.identity_pose(), p)
    S, T = r["sil"], r["t_final"]
    np.testing.assert_allclose(S + T, 1.0, atol=1e-12)
    assert S.min() >= 0 and S.max() <= 1
    assert T.min() >= p.t_min
    z = g.means[:, 2].astype(float)
    assert np.all(r["depth"] <= z.max() * S + 1e-12) and np.all(r["depth"] >= z.min() * S - 1e-12)
    for ch in range(3):
        assert np.all(r["rgb"][ch] <= g.rgb[:, ch].max() * S + 1e-12)
    assert r["amb"].mean() < 0.01


@pytest.mark.parametrize("seed", [0, 1])
def test_culled_equals_brute_force(seed):
    """Opacity-aware boxes are exact: culled and brute-force walks agree bit for bit."""
    rng = np.random.default_rng(seed)
    n = 200
    g = scenes.Gaussians(rng.uniform([-1, -1, 1], [1, 1, 3], (n, 3)).astype(np.float32),
                         rng.normal(size=(n, 4)).astype(np.float32),
                         rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32),
                         rng.normal(1.0, 1.0, n).astype(np.float32),
                         rng.uniform(0, 1, (n, 3)).astype(np.float32))
    cam = oracle.camera(50, 50, 31.5, 23.5, 64, 48)
    pose = scenes.perturb_pose(scenes.identity_pose(), rng, 3.0, 0.05)
    a = oracle.render(oracle_scene(g), cam, pose, oracle.Params())
    b = oracle.render(oracle_scene(g), cam, pose, oracle.Params(brute_force=True))
    for k in ("rgb", "depth", "sil", "t_final", "n_contrib", "amb"):
        assert np.array_equal(a[k], b[k]), k


def test_culled_equals_brute_force_cube():
    g, cam = scenes.cube_scene()
    oc = oracle_cam(cam)
    a = oracle.render(oracle_scene(g), oc, scenes.identity_pose(), oracle.Params())
    b = oracle.render(oracle_scene(g), oc, scenes.identity_pose(), oracle.Params(brute_force=True))
    for k in ("rgb", "depth", "sil", "t_final", "n_contrib"):
        assert np.array_equal(a[k], b[k]), k


def test_render_pixels_matches_full_frame():
    g, cam = scenes.cube_scene()
    oc = oracle_cam(cam)
    full = oracle.render(oracle_scene(g), oc, scenes.identity_pose(), oracle.Params())
    pix = np.random.default_rng(3).choice(cam.width * cam.height, 500, replace=False)
    sub = oracle.render_pixels(oracle_scene(g), oc, scenes.identity_pose(), oracle.Params(), pix)
    assert np.array_equal(sub["sil"], full["sil"].reshape(-1)[pix])
    assert np.array_equal(sub["depth"], full["depth"].reshape(-1)[pix])
    assert np.array_equal(sub["rgb"], full["rgb"].reshape(3, -1)[:, pix].T)


def test_isotropic_is_rotation_invariant(rng):
    """Equal scales (the isotropic Eq. 1): the image does not depend on the quaternion
    and the quaternion gradient is zero."""
    n = 30
    means = rng.uniform([-1, -1, 1.5], [1, 1, 3], (n, 3))
    ls = np.repeat(rng.normal(-3.2, 0.3, (n, 1)), 3, axis=1)
    logit, rgb = rng.normal(size=n), rng.uniform(size=(n, 3))
    cam = oracle.camera(60, 60, 23.5, 17.5, 48, 36)
    p = oracle.Params()
    r1 = oracle.render(oracle.Scene(means, rng.normal(size=(n, 4)), ls, logit, rgb), cam, scenes.identity_pose(), p)
    q2 = rng.normal(size=(n, 4))
    sc2 = oracle.Scene(means, q2, ls, logit, rgb)
    r2 = oracle.render(sc2, cam, scenes.identity_pose(), p)
    for k in ("rgb", "depth", "sil"):
        np.testing.assert_allclose(r1[k], r2[k], atol=1e-12)
    w = rng.normal(size=(5, 36, 48))
    b = oracle.backward(sc2, cam, scenes.identity_pose(), p, w[:3], w[3], w[4])
    assert np.abs(b["grads"][:, 3:7]).max() < 1e-9 * max(1.0, np.abs(b["grads"]).max())


# ----------------------------------------------------------------------------- gradients

def _tiny_scene(seed, n=6):
    rng = np.random.default_rng(seed)
    means = rng.uniform([-0.5, -0.4, 1.5], [0.5, 0.4, 2.5], (n, 3))
    return oracle.Scene(means, rng.normal(size=(n, 4)), rng.normal(-2.6, 0.3, (n, 3)),
                        rng.normal(0.5, 1.0, n), rng.uniform(size=(n, 3))), rng


def _functional(sc, cam, pose, p, w):
    r = oracle.render(sc, cam, pose, p)
    return (np.sum(w[:3] * r["rgb"]) + np.sum(w[3] * r["depth"]) + np.sum(w[4] * r["sil"]))


def _with(sc, name, i, k, val):
    arrs = {a: getattr(sc, a).copy() for a in ("means", "quats", "log_scales", "logits", "rgb")}
    if name == "logits":
        arrs[name][i] = val
    else:
        arrs[name][i, k] = val
    return oracle.Scene(**arrs)


@pytest.mark.parametrize("seed,jac_clip", [(0, 1.3), (1, 1.3), (2, 1.3), (3, 0.35)])
def test_backward_matches_finite_differences(seed, jac_clip):
    """Hand-derived reverse compositing and chain rule vs central finite differences of
    F = sum_p w . (C, D, S) with random weights, thresholds off (smooth maps), FP64.  The
    last case clamps the Jacobian's tangent for most Gaussians (no gradient through a
    clamped coordinate, the 1 / z factors still differentiated)."""
    sc, rng = _tiny_scene(seed)
    cam = oracle.camera(40, 40, 11.5, 8.5, 24, 18)
    pose = scenes.perturb_pose(scenes.identity_pose(), rng, 4.0, 0.05)
    p = _smooth_params(dilation=0.1 * seed, jac_clip=jac_clip)
    R0, t0 = scenes.pose_rt(pose)
    xc = sc.means @ R0.T + t0
    clamped = (np.abs(xc[:, 0] / xc[:, 2]) > jac_clip * 12 / 40) | (np.abs(xc[:, 1] / xc[:, 2]) > jac_clip * 9 / 40)
    assert clamped.sum() >= (3 if jac_clip < 1 else 0)
    w = rng.normal(size=(5, 18, 24))
    b = oracle.backward(sc, cam, pose, p, w[:3], w[3], w[4])
    g = b["grads"]
    cols = [("means", 3, 0), ("quats", 4, 3), ("log_scales", 3, 7), ("logits", 1, 10), ("rgb", 3, 11)]
    fd = np.zeros_like(g)
    for i in range(sc.n):
        for name, width, off in cols:
            for k in range(width):
                x0 = getattr(sc, name)[i] if name == "logits" else getattr(sc, name)[i, k]
                h = 1e-6 * max(1.0, abs(x0))
                fp = _functional(_with(sc, name, i, k, x0 + h), cam, pose, p, w)
                fm = _functional(_with(sc, name, i, k, x0 - h), cam, pose, p, w)
                fd[i, off + k] = (fp - fm) / (2 * h)
    scale = np.abs(fd).max()
    assert np.abs(g - fd).max() <= 1e-6 * scale, np.abs(g - fd).max() / scale
    # pose: left rotation perturbation and translation
    R, t = scenes.pose_rt(pose)
    fdp = np.zeros(6)
    h = 1e-6
    for k in range(6):
        vals = []
        for sgn in (1, -1):
            if k < 3:  # rotation about the camera centre: x_c -> Exp(e) x_c
                e = np.zeros(3)
                e[k] = sgn * h
                Re = Rotation.from_rotvec(e).as_matrix()
                P = scenes.pose_from_rt(Re @ R, Re @ t)
            else:
                tt = t.copy()
                tt[k - 3] += sgn * h
                P = scenes.pose_from_rt(R, tt)
            vals.append(_functional(sc, cam, P, p, w))
        fdp[k] = (vals[0] - vals[1]) / (2 * h)
    assert np.abs(b["pose6"] - fdp).max() <= 1e-6 * np.abs(fdp).max()


def test_backward_screen_space_fd():
    """The per-Gaussian screen-space gradient (d mu', d conic, d o, d rgb, d z) checked
    by perturbing a single Gaussian's colour / opacity through finite differences."""
    sc, rng = _tiny_scene(5)
    cam = oracle.camera(40, 40, 11.5, 8.5, 24, 18)
    p = _smooth_params()
    w = rng.normal(size=(5, 18, 24))
    b = oracle.backward(sc, cam, scenes.identity_pose(), p, w[:3], w[3], w[4])
    # rgb enters only through Eq. 2: d F / d rgb = screen-space rgb gradient
    np.testing.assert_allclose(b["grads"][:, 11:14], b["screen"][:, 6:9], rtol=0, atol=0)
    o = 1 / (1 + np.exp(-sc.logits))
    np.testing.assert_allclose(b["grads"][:, 10], b["screen"][:, 5] * o * (1 - o), rtol=1e-13)


def test_pose_gradient_equals_map_gradient_sums():
    """Moving the camera is moving the map: dL/dt = R sum_i dL/dmu_i.  Rotating every
    mean and covariance by delta about the world origin equals turning the camera by
    phi = R delta about its centre plus the translation change -phi x t, so
    R^T (dL/dtheta - t x dL/dt) is the map-rotation derivative (Sec. II-A x_c = R x + t),
    with the default thresholds on."""
    g, cam = scenes.cube_scene()
    sc, oc = oracle_scene(g), oracle_cam(cam)
    rng = np.random.default_rng(11)
    pose = scenes.perturb_pose(scenes.identity_pose(), rng, 2.0, 0.03)
    R, t = scenes.pose_rt(pose)
    w = rng.normal(size=(5, cam.height, cam.width))
    b = oracle.backward(sc, oc, pose, oracle.Params(), w[:3], w[3], w[4])
    gm, gq = b["grads"][:, 0:3], b["grads"][:, 3:7]
    np.testing.assert_allclose(b["pose6"][3:], R @ gm.sum(0), rtol=1e-9, atol=1e-9 * np.abs(b["pose6"]).max())
    # world rotation by delta: d x_i = delta x x_i, d q_i = 1/2 (0, delta) (x) q_i
    lhs = np.zeros(3)
    for k in range(3):
        e = np.eye(3)[k]
        dx = np.cross(e, sc.means)
        qw, qv = sc.quats[:, 0], sc.quats[:, 1:]
        dq = 0.5 * np.concatenate([(-(qv @ e))[:, None], qw[:, None] * e[None, :] + np.cross(e, qv)], axis=1)
        lhs[k] = np.sum(dx * gm) + np.sum(dq * gq)
    rhs = R.T @ (b["pose6"][:3] - np.cross(t, b["pose6"][3:]))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-8, atol=1e-9 * np.abs(b["pose6"]).max())


# ----------------------------------------------------------------------------- loss

def test_loss_worked_example():
    gold = json.load(open(os.path.join(GOLDEN, "loss_worked_example.json")))
    W, H = gold["width"], gold["height"]
    cam = oracle.camera(1, 1, 0, 0, W, H)
    p = oracle.Params(**gold["params"])
    rgb = np.array(gold["rgb"]).reshape(3, H, W)
    rgb_t = np.array(gold["rgb_t"]).reshape(3, H, W)
    out = oracle.loss(cam, p, rgb, np.array(gold["depth"]), np.array(gold["sil"]), rgb_t,
                      np.array(gold["depth_t"]), np.array(gold["prior"]))
    assert out["loss"] == pytest.approx(gold["loss"], abs=1e-12)
    np.testing.assert_allclose(out["d_rgb"].reshape(3, W), np.array(gold["d_rgb"]).reshape(3, W), atol=0)
    np.testing.assert_allclose(out["d_depth"].reshape(W), gold["d_depth"], atol=0)
    np.testing.assert_allclose(out["d_sil"].reshape(W), gold["d_sil"], atol=1e-15)


def test_loss_gradient_is_its_derivative(rng):
    """Upstream gradients = central differences of the loss w.r.t. each rendered value
    (away from L1 kinks and the silhouette threshold)."""
    W, H = 7, 5
    cam = oracle.camera(1, 1, 0, 0, W, H)
    p = oracle.Params()
    rgb, rgb_t = rng.uniform(size=(3, H, W)), rng.uniform(size=(3, H, W))
    depth, depth_t = rng.uniform(1, 3, (H, W)), rng.uniform(1, 3, (H, W))
    depth_t[0, :3] = 0
    prior = depth_t * 1.1
    prior[1, :2] = 0
    sil = np.where(rng.uniform(size=(H, W)) < 0.6, 0.995, 0.5)
    base = oracle.loss(cam, p, rgb, depth, sil, rgb_t, depth_t, prior)
    h = 1e-7
    for name, arr, grad in (("rgb", rgb, base["d_rgb"]), ("depth", depth, base["d_depth"]),
                            ("sil", sil, base["d_sil"])):
        flat = arr.reshape(-1)
        for j in range(flat.size):
            old = flat[j]
            vals = []
            for s in (h, -h):
                flat[j] = old + s
                args = dict(rgb=rgb, depth=depth, sil=sil)
                vals.append(oracle.loss(cam, p, args["rgb"], args["depth"], args["sil"], rgb_t, depth_t, prior)["loss"])
            flat[j] = old
            assert (vals[0] - vals[1]) / (2 * h) == pytest.approx(grad.reshape(-1)[j], abs=1e-6), (name, j)


# ----------------------------------------------------------------------------- pose update

def test_adam_first_steps_are_lr_sized():
    """Bias-corrected Adam moves each coordinate by lr sign(g) on its first step and on
    every step of a constant gradient (|g| >> eps), in both decoupled blocks."""
    p = oracle.Params(lr_rot=1e-3, lr_trans=5e-3)
    pose = scenes.identity_pose()
    state = np.zeros(16)
    g = np.array([0.0, 0.0, 3.0, -2.0, 0.5, 7.0])
    new, state = oracle.adam_step(pose, state, g, p)
    np.testing.assert_allclose(new[4:], -5e-3 * np.sign(g[3:]), rtol=1e-7)
    # rotation: Exp(-lr sign(g)) about z, on the left of the identity
    ang = 2 * np.arccos(np.clip(new[0], -1, 1))
    assert ang == pytest.approx(1e-3, rel=1e-6)
    assert new[3] < 0 and abs(new[1]) < 1e-15 and abs(new[2]) < 1e-15
    new2, state = oracle.adam_step(new, state, g, p)
    R1, t1 = scenes.pose_rt(new)
    R2, t2 = scenes.pose_rt(new2)
    rel = Rotation.from_matrix(R2 @ R1.T).as_rotvec()
    np.testing.assert_allclose(rel, [0, 0, -1e-3], atol=1e-12)
    # the camera centre moves by the translation step expressed in the new camera frame
    c1, c2 = -R1.T @ t1, -R2.T @ t2
    np.testing.assert_allclose(R2 @ (c2 - c1), 5e-3 * np.sign(g[3:]), rtol=1e-6)
    assert state[12] == 2


def test_adam_blocks_are_decoupled():
    """The rotation block turns the camera about its own centre (a pure rotation step
    leaves the centre where it was); the translation block moves the centre without
    turning the camera; neither block's step depends on the other block's gradient."""
    p = oracle.Params()
    pose = scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(0), 3.0, 0.4)
    R0, t0 = scenes.pose_rt(pose)
    rot_only, _ = oracle.adam_step(pose, np.zeros(16), np.array([1.0, -2, 3, 0, 0, 0]), p)
    R1, t1 = scenes.pose_rt(rot_only)
    np.testing.assert_allclose(-R1.T @ t1, -R0.T @ t0, atol=1e-14)
    assert np.linalg.norm(Rotation.from_matrix(R1 @ R0.T).as_rotvec()) > 1e-3
    trans_only, _ = oracle.adam_step(pose, np.zeros(16), np.array([0.0, 0, 0, 4, 5, -6]), p)
    np.testing.assert_allclose(trans_only[:4], pose[:4], atol=0)
    a, _ = oracle.adam_step(pose, np.zeros(16), np.array([1.0, -2, 3, 4, 5, 6]), p)
    b, _ = oracle.adam_step(pose, np.zeros(16), np.array([1.0, -2, 3, -40, 0.5, 60]), p)
    c, _ = oracle.adam_step(pose, np.zeros(16), np.array([-9.0, 2, 0.3, 4, 5, 6]), p)
    np.testing.assert_allclose(a[:4], b[:4], atol=0)
    for P in (a, c):  # same translation gradients: the centre moves the same distance
        R, t = scenes.pose_rt(P)
        assert np.linalg.norm(-R.T @ t + R0.T @ t0) == pytest.approx(np.sqrt(3) * p.lr_trans, rel=1e-6)


def test_adam_converges_on_quadratic():
    """Minimising |t - t*|^2 + |log(R R*^T)|^2 by the decoupled steps reaches the minimum."""
    rng = np.random.default_rng(2)
    target = scenes.perturb_pose(scenes.identity_pose(), rng, 10.0, 0.2)
    Rt, tt = scenes.pose_rt(target)
    p = oracle.Params(lr_rot=5e-3, lr_trans=5e-3)
    pose, state = scenes.identity_pose(), np.zeros(16)
    for _ in range(600):
        R, t = scenes.pose_rt(pose)
        # left-perturbation gradient of |log(R Rt^T)|^2 is 2 log(R Rt^T)
        g_rot = 2 * Rotation.from_matrix(R @ Rt.T).as_rotvec()
        pose, state = oracle.adam_step(pose, state, np.concatenate([g_rot, 2 * (t - tt)]), p)
    R, t = scenes.pose_rt(pose)
    assert np.linalg.norm(t - tt) < 5e-3
    assert np.linalg.norm(Rotation.from_matrix(R @ Rt.T).as_rotvec()) < 5e-3


def test_oracle_tracking_reduces_pose_error():
    """Sanity (not parity): decoupled tracking on the cube scene moves the pose toward
    the one the target was rendered from."""
    g, cam = scenes.cube_scene()
    sc, oc = oracle_scene(g), oracle_cam(cam)
    rng = np.random.default_rng(0)
    gt = scenes.identity_pose()
    start = scenes.perturb_pose(gt, rng, 2.0, 0.03)
    p = oracle.Params(lr_rot=2e-3, lr_trans=2e-3)
    tgt = oracle.render(sc, oc, gt, p)
    pose, state = start.copy(), np.zeros(16)

    def err(P):
        R, t = scenes.pose_rt(P)
        R0, t0 = scenes.pose_rt(gt)
        return np.linalg.norm(t - t0), np.linalg.norm(Rotation.from_matrix(R @ R0.T).as_rotvec())

    e0 = err(pose)
    for _ in range(15):
        r = oracle.render(sc, oc, pose, p)
        L = oracle.loss(oc, p, r["rgb"], r["depth"], r["sil"], tgt["rgb"], tgt["depth"], None)
        b = oracle.backward(sc, oc, pose, p, L["d_rgb"], L["d_depth"], L["d_sil"])
        pose, state = oracle.adam_step(pose, state, b["pose6"], p)
    e1 = err(pose)
    assert e1[0] < 0.8 * e0[0] and e1[1] < 0.8 * e0[1]
