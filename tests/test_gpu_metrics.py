"""Evaluation kernels (gs_image_metrics, gs_msssim) against the metric oracle through
the C ABI.  The image sums are FP64 in a fixed order (relative 1e-9 of the oracle's);
MS-SSIM takes its local statistics in FP32 centred on the window's middle pixel and
sums in FP64 (absolute 2e-5 on each channel's value)."""
import numpy as np
import pytest
import torch

from oracle import metrics as omx
from paper_2408_05635_gb300 import gs, scenes

pytestmark = pytest.mark.gpu


def _pair(W, H, seed, noise):
    cam = scenes.Cam(0.8 * W, 0.8 * W, (W - 1) / 2, (H - 1) / 2, W, H)
    pose = scenes.look_at((2.5, 1.5, 0.8), (0.1, -0.05, 1.0))
    rgb, depth = scenes.raycast_room(pose, cam, seed=seed)
    rng = np.random.default_rng(seed)
    rgb2 = np.clip(rgb + rng.normal(0, noise, rgb.shape), 0, 1).astype(np.float32)
    depth2 = (depth * (1 + rng.normal(0, 0.01, depth.shape))).astype(np.float32)
    return np.ascontiguousarray(rgb), np.ascontiguousarray(depth), rgb2, depth2


@pytest.mark.parametrize("W,H", [(640, 480), (333, 257)])
def test_image_sums_and_msssim_match_oracle(W, H):
    rgb, depth, rgb2, depth2 = _pair(W, H, seed=W, noise=0.04)
    t = [torch.from_numpy(a).cuda() for a in (rgb2, depth2, rgb, depth)]
    sums = torch.zeros(4, dtype=torch.float64, device="cuda")
    gs.gs_image_metrics(t[0], t[1], t[2], t[3], sums)
    ms = torch.zeros(4, dtype=torch.float64, device="cuda")
    gs.gs_msssim(t[0], t[2], W, H, ms)
    torch.cuda.synchronize()
    ref = omx.image_sums(rgb2, depth2, rgb, depth)
    np.testing.assert_allclose(sums.cpu().numpy(), ref, rtol=1e-9)
    o = omx.ms_ssim(rgb2, rgb)
    got = ms.cpu().numpy()
    print(f"{W}x{H}: MS-SSIM gpu {got[0]:.6f} oracle {o['ms_ssim']:.6f}")
    np.testing.assert_allclose(got[1:], o["per_channel"], atol=2e-5)
    assert got[0] == pytest.approx(o["ms_ssim"], abs=2e-5)
    assert 0.0 < got[0] < 1.0


def test_msssim_of_identical_images_is_one():
    rgb, _, _, _ = _pair(400, 300, seed=3, noise=0.0)
    x = torch.from_numpy(rgb).cuda()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    gs.gs_msssim(x, x, 400, 300, out)
    np.testing.assert_allclose(out.cpu().numpy(), 1.0, atol=1e-12)
