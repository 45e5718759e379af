"""gs_render_static: the single-view render that allocates nothing, its scratch being a
static device array of the library.  It is meant for callers that cannot allocate
device memory where they render (a plugin inside a host application that owns the
memory pool, or code that must not call cudaMalloc / cudaFree).  Its outputs must match
the workspace-based gs_project + gs_forward on the same inputs, on consecutive calls
(the array keeps the previous call's contents, so a second call checks the clearing).
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2408_05635_gb300 import gs, scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4  # the image tolerance of the parity tests


def _inputs(seed, n=2000):
    g, cam = scenes.cube_scene(n=n, seed=seed)
    pose = scenes.perturb_pose(scenes.identity_pose(), np.random.default_rng(seed), 1.5, 0.02)
    rng = np.random.default_rng(seed + 100)
    t_rgb = rng.uniform(size=(3, cam.height, cam.width)).astype(np.float32)
    t_depth = rng.uniform(1.0, 3.0, size=(cam.height, cam.width)).astype(np.float32)
    return g, cam, pose, t_rgb, t_depth


def _workspace_render(g, cam, pose, t_rgb, t_depth):
    R = gs.Rasterizer(gs.Config())
    gt = gs.GaussianTensors.from_numpy(g)
    poses = torch.tensor(np.asarray(pose)[None], dtype=torch.float64, device="cuda")
    prob = R.plan(gt, [cam], poses)
    tt = (torch.tensor(t_rgb.reshape(-1), device="cuda"), torch.tensor(t_depth.reshape(-1), device="cuda"), None)
    out = R.render(prob, gt, poses, targets=tt)
    R.sync()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _static_render(g, cam, pose, t_rgb, t_depth):
    gt = gs.GaussianTensors.from_numpy(g)
    pose_t = torch.tensor(np.asarray(pose), dtype=torch.float64, device="cuda")
    P = cam.width * cam.height
    out = {"rgb": torch.empty(3 * P, device="cuda"), "depth": torch.empty(P, device="cuda"),
           "sil": torch.empty(P, device="cuda"), "loss": torch.empty(1, dtype=torch.float64, device="cuda")}
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    tr = torch.tensor(t_rgb.reshape(-1), device="cuda")
    td = torch.tensor(t_depth.reshape(-1), device="cuda")
    targets = gs.gs_targets(tr.data_ptr(), td.data_ptr(), None)
    gs.gs_render_static(gs.Config().c(), gt.c(), gs.cameras_c([cam])[0], pose_t, targets, out["rgb"], out["depth"],
                        out["sil"], out["loss"], err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_static_render_matches_workspace_render_twice():
    for seed in (0, 1):  # two calls in a row, different scenes: nothing stale may leak through
        args = _inputs(seed)
        ref = _workspace_render(*args)
        got = _static_render(*args)
        for k in ("rgb", "depth", "sil"):
            assert np.abs(got[k] - ref[k]).max() <= IMG_TOL, k
        assert got["loss"][0] == pytest.approx(ref["loss"][0], rel=2e-4)


def test_static_render_rejects_oversized_requests():
    g, cam, pose, t_rgb, t_depth = _inputs(0, n=100)
    big = scenes.Cam(100.0, 100.0, 400.0, 300.0, 800, 600)  # 480k pixels > the 307,200 limit
    gt = gs.GaussianTensors.from_numpy(g)
    pose_t = torch.tensor(np.asarray(pose), dtype=torch.float64, device="cuda")
    with pytest.raises(gs.GsError) as e:
        gs.gs_render_static(gs.Config().c(), gt.c(), gs.cameras_c([big])[0], pose_t)
    assert e.value.status == 1
