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
