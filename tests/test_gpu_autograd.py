"""torch.autograd wrapper: gradients of a scalar of the rendered maps, through
gs_backward, against the FP64 oracle's gradients for the same upstream maps; the
recomputing backward equals the stored one."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import assert_grads_close, ocam, params_pair
from paper_2408_05635_gb300 import autograd, gs, scenes

pytestmark = pytest.mark.gpu

NAMES = [("means", 0, 3), ("quats", 3, 7), ("log_scales", 7, 10), ("logits", 10, 11), ("rgb", 11, 14)]


def _leaf(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda", requires_grad=True)


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_matches_oracle(recompute):
    g, cam = scenes.cube_scene(n=1500, seed=4)
    pose = scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(2), 1.0, 0.02)
    gcfg, op = params_pair()
    R = gs.Rasterizer(gcfg)
    leaves = [_leaf(a) for a in g.arrays()]
    poses = torch.tensor(np.asarray(pose)[None], dtype=torch.float64, device="cuda")
    tangent = torch.zeros(1, 6, dtype=torch.float64, device="cuda", requires_grad=True)
    rgb, depth, sil = autograd.render(R, *leaves, [cam], poses, tangent, recompute=recompute)
    H, W = cam.height, cam.width
    ref = oracle.render(oracle.Scene(*g.arrays()), ocam(cam), pose, op)
    rng = np.random.default_rng(9)
    w = rng.normal(size=(5, H, W))
    w[:, ref["amb"]] = 0.0  # same upstream on both sides, ambiguous pixels excluded
    wt = [torch.tensor(x.reshape(-1), dtype=torch.float32, device="cuda") for x in (w[:3], w[3], w[4])]
    loss = (rgb * wt[0]).sum() + (depth * wt[1]).sum() + (sil * wt[2]).sum()
    loss.backward()
    ob = oracle.backward(oracle.Scene(*g.arrays()), ocam(cam), pose, op, w[:3], w[3], w[4])
    for leaf, (name, lo, hi) in zip(leaves, NAMES):
        assert_grads_close(leaf.grad.cpu().numpy().reshape(g.n, -1), ob["grads"][:, lo:hi], what=name)
    assert_grads_close(tangent.grad.cpu().numpy()[0], ob["pose6"], what="pose")


def _apply_tangent(pose, theta, shift):
    """The pose after turning the camera about its own centre by Exp(theta) and shifting
    it by `shift` in the camera frame (x_c <- Exp(theta) x_c + shift): the two blocks
    whose gradient autograd.render returns through pose_tangent."""
    from scipy.spatial.transform import Rotation
    Rm, t = scenes.pose_rt(pose)
    E = Rotation.from_rotvec(np.asarray(theta, np.float64)).as_matrix()
    return scenes.pose_from_rt(E @ Rm, E @ t + np.asarray(shift, np.float64))


def test_autograd_matches_finite_differences():
    """Finite differences through the wrapper itself.  Thresholds off (alpha_min = t_min = 0,
    alpha_max = 1) so the maps are smooth in every parameter; L is a fixed random linear
    function of the rendered colour, depth and silhouette, summed in FP64 (|L| is about 50).
    For each parameter group and each pose block, a random direction v and the points
    x-, x0, x+ = x - h v, x, x + h v as rendered (FP32 for the parameters, so their rounding
    is no error of the check): the change L(x+) - L(x-) must equal the path integral of the
    autograd gradient, taken by Simpson's rule from the gradients at the three points
    (error O(h^5), so steps can be large enough that the FP32 noise of L, about 1e-4, is
    below 1e-3 of the change).  Means move in the image plane (v with no component along
    the camera axis) and the camera turns by 2e-4 rad at most: a larger change of depth
    would let two Gaussians swap their front-to-back order, a jump of L that no gradient
    describes.  The translation block moves every depth alike and so covers d/dz.  With
    the FP64 oracle in place of the GPU the same check agrees to 1e-3 (quaternions) and
    below 1e-5 elsewhere; bound 1e-2 relative."""
    g, _ = scenes.cube_scene(n=120, seed=11)
    g.log_scales += np.float32(1.0)  # footprints of 2 to 3 px at this focal length
    cam = scenes.Cam(56.0, 56.0, 31.5, 23.5, 64, 48)
    H, W = cam.height, cam.width
    R = gs.Rasterizer(gs.Config(alpha_min=0.0, t_min=0.0, alpha_max=1.0))
    pose = scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(2), 1.0, 0.02)
    rng = np.random.default_rng(3)
    w = [torch.tensor(rng.normal(size=k * H * W), dtype=torch.float64, device="cuda") for k in (3, 1, 1)]

    def run(arrays, pose_np, grad=True):
        """L at (arrays, pose) and, with grad, its gradients: five parameter groups and
        the pose 6-vector."""
        leaves = [_leaf(a) for a in arrays]
        poses = torch.tensor(np.asarray(pose_np)[None], dtype=torch.float64, device="cuda")
        tangent = torch.zeros(1, 6, dtype=torch.float64, device="cuda", requires_grad=True)
        with torch.set_grad_enabled(grad):
            outs = autograd.render(R, *leaves, [cam], poses, tangent)
            L = sum((o.double() * wk).sum() for o, wk in zip(outs, w))
        if not grad:
            return float(L), None, None
        L.backward()
        return (float(L.detach()), [leaf.grad.cpu().numpy().astype(np.float64) for leaf in leaves],
                tangent.grad.cpu().numpy()[0])

    def check(what, lm, lp, dm, d0, dp):
        simpson = (dm + 4.0 * d0 + dp) / 6.0
        assert abs((lp - lm) - simpson) <= 1e-2 * abs(simpson), f"{what}: dL {lp - lm:.6e}, autograd {simpson:.6e}"

    base = [np.asarray(a, np.float32) for a in g.arrays()]
    _, g0, p0 = run(base, pose)
    rz = scenes.pose_rt(pose)[0][2]  # camera axis in world coordinates
    steps = {"means": 2e-3, "quats": 2e-2, "log_scales": 2e-2, "logits": 2e-2, "rgb": 5e-2}
    for k, (name, _, _) in enumerate(NAMES):
        v = rng.normal(size=base[k].shape)
        if name == "means":
            v -= np.outer(v @ rz, rz)
        plus, minus = list(base), list(base)
        plus[k] = (base[k] + steps[name] * v).astype(np.float32)
        minus[k] = (base[k] - steps[name] * v).astype(np.float32)
        dx = plus[k].astype(np.float64) - minus[k].astype(np.float64)
        lp, gp, _ = run(plus, pose)
        lm, gm, _ = run(minus, pose)
        check(name, lm, lp, float((gm[k] * dx).sum()), float((g0[k] * dx).sum()), float((gp[k] * dx).sum()))
    for block, h in (("rotation", 2e-4), ("translation", 2e-3)):
        d = np.zeros(6)
        off = 0 if block == "rotation" else 3
        d[off:off + 3] = h * rng.normal(size=3)
        pp, pm = _apply_tangent(pose, d[:3], d[3:]), _apply_tangent(pose, -d[:3], -d[3:])
        lp, _, qp = run(base, pp)
        lm, _, qm = run(base, pm)
        check(f"pose {block}", lm, lp, float(qm @ (2 * d)), float(p0 @ (2 * d)), float(qp @ (2 * d)))
