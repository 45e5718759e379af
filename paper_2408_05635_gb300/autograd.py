"""torch.autograd wrapper of the rasterizer: forward = gs_project + gs_forward, backward =
gs_backward, every step in the CUDA library.

``render(...)`` returns the concatenated planar colour (3 x H x W per view), depth and
silhouette (H x W per view) of every view.  Gradients reach the Gaussian parameters and,
through ``pose_tangent`` (n_views x 6, float64, its value is not used), the poses: the
gradient of ``pose_tangent`` is dL/d(theta, t) for a rotation of each camera about its own
centre (x_c <- Exp(theta) x_c) and a shift (x_c <- x_c + t), the blocks the decoupled
tracking update of Sec. III-B optimises.

With ``recompute=True`` the backward re-runs the projection, the per-tile binning and
sort and the forward compositing before it walks back, instead of relying on the state
the forward left in the workspace: a mapping window can then render view after view
through one workspace and still back-propagate every view.
"""
from __future__ import annotations

import torch

from . import gs


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, quats, log_scales, logits, rgb, pose_tangent, rast, cams, poses, recompute):
        g = gs.GaussianTensors(means.detach().contiguous(), quats.detach().contiguous(),
                               log_scales.detach().contiguous(), logits.detach().contiguous(),
                               rgb.detach().contiguous())
        poses = poses.detach().contiguous()
        prob = rast.plan(g, cams, poses)
        out = rast.render(prob, g, poses)
        ctx.rast, ctx.cams, ctx.prob, ctx.recompute = rast, cams, prob, recompute
        ctx.token = id(out["rgb"])
        rast._autograd_token = ctx.token
        ctx.save_for_backward(means, quats, log_scales, logits, rgb, poses)
        return out["rgb"], out["depth"], out["sil"]

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_sil):
        means, quats, log_scales, logits, rgb, poses = ctx.saved_tensors
        rast = ctx.rast
        g = gs.GaussianTensors(means.detach().contiguous(), quats.detach().contiguous(),
                               log_scales.detach().contiguous(), logits.detach().contiguous(),
                               rgb.detach().contiguous())
        if ctx.recompute or getattr(rast, "_autograd_token", None) != ctx.token:
            rast.render(ctx.prob, g, poses, images=False)  # rebuild lists and transmittance
        P = _pixels(ctx.cams)
        ups = tuple(g.means.new_zeros(k * P) if u is None else u.float().contiguous()
                    for u, k in ((d_rgb, 3), (d_depth, 1), (d_sil, 1)))
        b = rast.backward(g, upstream=ups, params=True, pose=True, n_views=len(ctx.cams))
        rast._autograd_token = None
        G = b["grads"]
        cast = lambda x, like: x.to(like.dtype)
        return (cast(G["means"], means), cast(G["quats"], quats), cast(G["log_scales"], log_scales),
                cast(G["logits"], logits), cast(G["rgb"], rgb), b["pose_grad"], None, None, None, None)


def _pixels(cams) -> int:
    return sum(int(c.width) * int(c.height) for c in cams)


def render(rast: gs.Rasterizer, means, quats, log_scales, logits, rgb, cams, poses, pose_tangent=None,
           recompute: bool = False):
    """Differentiable render of len(cams) views.  poses: n_views x 7 float64 CUDA tensor
    (world->camera [qw, qx, qy, qz, tx, ty, tz]); pose_tangent: optional n_views x 6 float64
    tensor with requires_grad to receive the pose gradient."""
    if pose_tangent is None:
        pose_tangent = torch.zeros(len(cams), 6, dtype=torch.float64, device=means.device)
    return _Rasterize.apply(means, quats, log_scales, logits, rgb, pose_tangent, rast, list(cams), poses,
                            recompute)
