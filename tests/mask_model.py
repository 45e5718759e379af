"""The share of pixels the oracle's ambiguity mask flags, predicted from its margins by
two closed forms (restated here, independent of the oracle's own code):
  - a Gaussian's alpha lies within a relative margin m of alpha_min on an annulus of area
    4 pi m sqrt(det Sigma') pixels: ln alpha = ln o - d^2 / 2, so the annulus is
    |d^2 - D^2| <= 2m around the support ellipse d^2 = D^2 (area pi d^2 sqrt(det Sigma'));
  - a walk that stops on t_min lands within a relative margin e of t_min, on either side,
    with probability about 2 e / s for a last step of size s = -ln(1 - alpha) in log
    transmittance.
Both are upper bounds of the flagged shares (occlusion and the alpha_min effect gate only
remove flags); the bounds add three Poisson standard deviations and one pixel.  Used by
the CPU pins of the mask and by the GPU parity tests in place of a fixed share.
"""
import numpy as np

import oracle
from paper_2408_05635_gb300 import scenes

U = 2.0 ** -24  # unit roundoff of binary32


def annulus_share(sc, cam, pose, op):
    """Expected share of pixels with an alpha within its margin of alpha_min: the sum
    over on-image Gaussians of 4 pi m sqrt(det Sigma'), m the margin averaged over the
    support ellipse (restated: the floor amb_alpha, or the exponent error 4u (|Q d| |mu'| +
    |terms|) + |Q d| dmu with dmu = (f / z)(1 + |x_c / z| + |y_c / z|) 2u (|m| + |t|)),
    counting the part of the annulus inside the image, over the pixel count."""
    pr = oracle.project(sc, oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height), pose, op)
    v = pr["valid"]
    mu, cov, conic, o, z = pr["mu"][v], pr["cov2"][v], pr["conic"][v], pr["opacity"][v], pr["z"][v]
    D2 = 2.0 * np.log(o / op.alpha_min)
    det = cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2
    L00 = np.sqrt(cov[:, 0])
    L10 = cov[:, 1] / L00
    L11 = np.sqrt(np.maximum(cov[:, 2] - L10 ** 2, 0.0))
    R, t = scenes.pose_rt(pose)
    m = sc.means[v]
    xc = m @ R.T + t
    dmu = max(cam.fx, cam.fy) / z * 2 * U * (np.linalg.norm(m, axis=1) + np.linalg.norm(t)) * (
        1 + np.abs(xc[:, 0] / z) + np.abs(xc[:, 1] / z))
    mu_mag = np.maximum(np.abs(mu[:, 0]), np.abs(mu[:, 1]))
    K = 32
    margin = np.zeros(len(o))
    inside = np.zeros(len(o))
    for a in np.linspace(0.0, 2 * np.pi, K, endpoint=False):
        wx, wy = np.cos(a) * np.sqrt(D2), np.sin(a) * np.sqrt(D2)
        dx, dy = L00 * wx, L10 * wx + L11 * wy  # a point of the support ellipse
        gx, gy = conic[:, 0] * dx + conic[:, 1] * dy, conic[:, 1] * dx + conic[:, 2] * dy
        grad = np.hypot(gx, gy)
        terms = np.abs(conic[:, 0] * dx * dx) + 2 * np.abs(conic[:, 1] * dx * dy) + np.abs(conic[:, 2] * dy * dy)
        margin += np.maximum(op.amb_alpha, 4 * U * (grad * mu_mag + terms) + grad * dmu) / K
        px, py = mu[:, 0] + dx, mu[:, 1] + dy
        inside += ((px > -0.5) & (px < cam.width - 0.5) & (py > -0.5) & (py < cam.height - 0.5)) / K
    count = (4.0 * np.pi * margin * np.sqrt(det) * inside).sum()
    return count / (cam.width * cam.height), count



def t_min_expectation(sc, cam, pose, op):
    """Expected number of pixels flagged for t_min: the sum over the pixels whose walk
    stops of min(1, 2 max(amb_t, eT) / s)."""
    ts = oracle.render_tstats(sc, oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height), pose, op)
    stops = ts["step"] > 0
    return float(np.minimum(1.0, 2.0 * np.maximum(op.amb_t, ts["eT"][stops]) / ts["step"][stops]).sum())


def mask_shares(sc, cam, pose, op, ref) -> dict:
    """Flagged shares by reason (ref: oracle.render of the same view) and their bounds."""
    npix = cam.width * cam.height
    bits = ref["amb_bits"]
    a_share, a_count = annulus_share(sc, cam, pose, op)
    t_count = t_min_expectation(sc, cam, pose, op)
    return {"all": float(ref["amb"].mean()),
            "alpha_min": float((bits & oracle.AMB_ALPHA_MIN).astype(bool).mean()),
            "alpha_min_bound": a_share + (3.0 * np.sqrt(a_count) + 1.0) / npix,
            "t_min": float((bits & oracle.AMB_T_MIN).astype(bool).mean()),
            "t_min_bound": (t_count + 3.0 * np.sqrt(t_count) + 1.0) / npix,
            "alpha_max": float((bits & oracle.AMB_ALPHA_MAX).astype(bool).mean())}
