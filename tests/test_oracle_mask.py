"""Pins of the oracle's two FP32-facing parts, checked without the CUDA path.

The depth key.  Eqs. 2-4 composite front to back, and the order is a discrete decision:
both implementations take it on one exactly specified FP32 key (depth_key in
gs_oracle.c).  Pinned here against the FP64 camera depth of the mean: the key is that
depth to within its rounding bound, and the key order is the FP64 order except for pairs
whose FP64 depths lie within the two keys' rounding bounds of each other.

The ambiguity mask.  Where an FP32 renderer may take another discrete decision than the
FP64 walk (an alpha within its margin of alpha_min, a transmittance within its margin of
t_min), the oracle flags the pixel and lists every outcome of it (render_alternatives).
  - Soundness: a render under the error model the mask assumes -- the pose rounded to
    FP32 as the GPU applies it, every footprint exponent moved by up to its modelled
    rounding error -- lands, at every pixel, within 1e-4 of the nominal outcome
    (unflagged pixels) or of one of the listed outcomes (flagged pixels).
  - Tightness: the share of pixels flagged is what the margins predict, from two closed
    forms restated here: a Gaussian's alpha lies within a relative margin m of alpha_min
    on an annulus of area 4 pi m sqrt(det Sigma') pixels (ln alpha = ln o - d^2 / 2, so
    the annulus is |d^2 - D^2| <= 2m around the support ellipse d^2 = D^2, of area
    pi d^2 sqrt(det Sigma')); and a walk that stops on t_min lands within a relative
    margin e of t_min, on either side, with probability about 2 e / s for a last step
    of size s = -ln(1 - alpha) in log transmittance.
"""
import numpy as np
import pytest

import mask_model
import oracle
from paper_2408_05635_gb300 import scenes

U = 2.0 ** -24  # unit roundoff of binary32


def _cam(c):
    return oracle.camera(c.fx, c.fy, c.cx, c.cy, c.width, c.height)


def _opaque_stacks():
    """Stacks of nearly opaque Gaussians (alpha 0.95 .. 0.99) over the cube scene: many
    pixels stop on t_min after few steps."""
    g, _ = scenes.cube_scene(n=600, seed=21)
    rng = np.random.default_rng(21)
    xy = rng.uniform(-0.45, 0.45, size=(24, 2))
    means, logits = [], []
    for s in range(24):
        for k in range(4):
            means.append([xy[s, 0] + rng.normal(0, 0.004), xy[s, 1] + rng.normal(0, 0.004), 1.2 + 0.05 * k])
            logits.append([6.0, 4.0, 5.0, 3.0][k])
    m = len(means)
    stack = [np.asarray(means, np.float32), rng.normal(size=(m, 4)).astype(np.float32),
             rng.normal(-3.2, 0.15, size=(m, 3)).astype(np.float32), np.asarray(logits, np.float32),
             rng.uniform(0, 1, size=(m, 3)).astype(np.float32)]
    return scenes.Gaussians(*(np.concatenate([a, b]) for a, b in zip(stack, g.arrays())))


def _cases():
    """(name, Gaussians, camera, pose): the small parity scenes, the near-opaque stacks
    and the 640 x 480 / 200k room tracking frame at its start pose."""
    out = []
    g, cam = scenes.cube_scene()
    out.append(("cube 160x120", g, cam, scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(5), 1.0,
                                                          0.02)))
    g, _ = scenes.cube_scene(n=600, seed=3)
    out.append(("ragged 37x23", g, scenes.Cam(40.0, 44.0, 18.3, 11.1, 37, 23),
                scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(5), 1.0, 0.02)))
    out.append(("opaque stacks 96x72", _opaque_stacks(), scenes.Cam(100.0, 100.0, 47.5, 35.5, 96, 72),
                scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(8), 0.5, 0.01)))
    # the tracking frame: the 200k-Gaussian room, its ground-truth camera and the start
    # pose 2 deg / 5 cm away
    g = scenes.room_scene(200_000, seed=0)
    start = scenes.perturb_pose(scenes.tracking_gt_pose(), np.random.default_rng(1), 2.0, 0.05)
    out.append(("room 640x480", g, scenes.TUM_CAM, start))
    return out


CASES = _cases()
IDS = [c[0] for c in CASES]


def _key_bound(means, pose):
    """Rounding bound of the FP32 depth key: the pose's rotation and translation rounded
    to FP32 (rotation entries from a normalised FP32 quaternion: a few units of roundoff
    each) and three rounded fused multiply-adds, all relative to |R_2k m_k| + |t_2|."""
    R, t = scenes.pose_rt(pose)
    return 16.0 * U * (np.abs(means) @ np.abs(R[2]) + abs(t[2]))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_depth_key_follows_the_exact_depth_order(case):
    name, g, cam, pose = case
    sc = oracle.Scene(*g.arrays())
    keys, z = oracle.depth_keys(sc, pose)
    b = _key_bound(sc.means, pose)
    # the key is the FP64 camera depth to within its rounding bound
    assert np.all(np.abs(keys.astype(np.float64) - z) <= b), np.abs(keys - z).max()
    # sorted by (key, index), no pair is out of FP64 order by more than both bounds:
    # z_j >= z_i - b_i - b_j for every i before j, i.e. the running maximum of z - b over
    # the prefix never exceeds z_j + b_j
    order = np.lexsort((np.arange(g.n), keys))
    zs, bs = z[order], b[order]
    prefix = np.maximum.accumulate(zs - bs)
    assert np.all(prefix[:-1] <= zs[1:] + bs[1:])
    # and the bound is tight enough to constrain the order: most neighbours in key order
    # are farther apart in FP64 depth than their two bounds
    assert (np.diff(zs) > bs[:-1] + bs[1:]).mean() > 0.5


def _max_err(a, b):
    """Max over colour, depth and silhouette of |a - b| per pixel."""
    return np.maximum(np.abs(a["rgb"] - b["rgb"]).max(axis=0),
                      np.maximum(np.abs(a["depth"] - b["depth"]), np.abs(a["sil"] - b["sil"])))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_mask_is_sound_under_the_fp32_error_model(case):
    name, g, cam, pose = case
    sc, oc, op = oracle.Scene(*g.arrays()), _cam(cam), oracle.Params()
    ref = oracle.render(sc, oc, pose, op)
    flagged = ref["amb"].ravel()
    pix = np.flatnonzero(flagged)
    alts = oracle.render_alternatives(sc, oc, pose, op, pix, max_alt=32)
    n_alt, A = alts["n_alt"], alts["alts"]
    resolved = n_alt > 0
    # the nominal outcome is one of the listed ones
    nom = np.stack([ref["rgb"][0].ravel()[pix], ref["rgb"][1].ravel()[pix], ref["rgb"][2].ravel()[pix],
                    ref["depth"].ravel()[pix], ref["sil"].ravel()[pix], ref["t_final"].ravel()[pix]], 1)
    for k in np.flatnonzero(resolved):
        assert np.abs(A[k, :n_alt[k]] - nom[k]).max(axis=1).min() < 1e-12
    for seed in range(3):
        q = oracle.render_perturbed(sc, oc, pose, op, seed, 1.0)
        err = _max_err(q, ref).ravel()
        bad = (err > 1e-4) & ~flagged
        assert not bad.any(), f"{name}: {bad.sum()} unflagged pixels moved by up to {err[bad].max():.2e}"
        got = np.stack([q["rgb"][0].ravel()[pix], q["rgb"][1].ravel()[pix], q["rgb"][2].ravel()[pix],
                        q["depth"].ravel()[pix], q["sil"].ravel()[pix]], 1)
        for k in np.flatnonzero(resolved):
            d = np.abs(A[k, :n_alt[k], :5] - got[k]).max(axis=1).min()
            assert d <= 1e-4, f"{name}: flagged pixel {pix[k]} is {d:.2e} from every listed outcome"


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_mask_share_is_what_its_margins_predict(case):
    """Upper bounds: the alpha_min share at most the annulus expectation (every annulus
    pixel counted, occlusion and the effect gate ignored) plus three Poisson standard
    deviations; the t_min share at most the sum of 2 max(amb_t, eT) / s over the pixels
    that stop, plus three standard deviations.  A wider margin anywhere breaks them."""
    name, g, cam, pose = case
    sc, op = oracle.Scene(*g.arrays()), oracle.Params()
    ref = oracle.render(sc, _cam(cam), pose, op)
    m = mask_model.mask_shares(sc, cam, pose, op, ref)
    assert m["alpha_min"] <= m["alpha_min_bound"], m
    assert m["t_min"] <= m["t_min_bound"], m
    print(f"{name}: " + ", ".join(f"{k} {v:.4%}" for k, v in m.items()))
