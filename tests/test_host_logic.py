"""Host logic of the sequence driver on the CPU, with the CUDA calls replaced by fakes:
slam.Tracker plans once per map, tunes the launch schedule on the first frame and again
once the map has more than doubled, re-plans with a larger pair capacity when the device
reports an overflow, and gives up after repeated overflows."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

from paper_2408_05635_gb300 import gs, slam

CAM = SimpleNamespace(fx=100.0, fy=100.0, cx=15.5, cy=11.5, width=32, height=24)


class FakeRasterizer:
    """Records what the tracker asks for instead of launching anything."""

    def __init__(self, config=None, device="cuda"):
        self.ctx = object()
        self.log = []

    def plan(self, g, cams, poses, margin=1.25):
        self.log.append(("plan", g.n, margin))
        return SimpleNamespace(pair_capacity=1000)

    def problem(self, n, cams, pair_capacity):
        self.log.append(("problem", n, pair_capacity))
        return SimpleNamespace(pair_capacity=pair_capacity)

    def workspace(self, prob):
        return None, 0

    def autotune(self, prob, g, poses, targets, pose_only=True, reps=10, stream=None):
        self.log.append(("autotune", g.n, pose_only, reps))
        return {"schedule": {"tile_w": 16, "tile_h": 16}, "timings_ms": []}

    @property
    def schedule(self):
        return {"tile_w": 16, "tile_h": 16}

    def close(self):
        pass


def _map(n):
    means = torch.zeros(n, 3)
    return SimpleNamespace(means=means, n=n, log_scales=torch.zeros(n, 3), isotropic=False, c=lambda: None)


@pytest.fixture
def fake(monkeypatch):
    status = []  # (status, n_pairs) the next gs_sync_status calls report
    monkeypatch.setattr(gs, "Rasterizer", FakeRasterizer)
    monkeypatch.setattr(gs, "gs_track_step", lambda *a, **k: None)

    def sync(ctx, stream=None):
        st, pairs = status.pop(0) if status else (0, 10)
        return st, SimpleNamespace(n_pairs=pairs)

    monkeypatch.setattr(gs, "gs_sync_status", sync)
    return status


def _frame():
    return torch.zeros(3, CAM.height, CAM.width), torch.ones(CAM.height, CAM.width)


def test_tracker_plans_and_tunes_per_map_size(fake):
    tr = slam.Tracker(CAM, 5, device="cpu", autotune_reps=3)
    start = torch.tensor([1.0, 0, 0, 0, 0, 0, 0], dtype=torch.float64)
    g1 = _map(1000)
    tr.track(g1, start, *_frame())
    tr.track(g1, start, *_frame())  # same map: neither planned nor tuned again
    assert [e[0] for e in tr.R.log] == ["plan", "autotune", "plan"]
    assert tr.R.log[1] == ("autotune", 1000, True, 3) and tr.tunes == 1
    # the tuning problem has twice the pair margin of the tracking problem
    assert tr.R.log[0][2] == pytest.approx(2 * tr.R.log[2][2])
    tr.track(_map(2000), start, *_frame())  # doubled, not more: re-planned only
    assert tr.tunes == 1 and tr.R.log[-1][:2] == ("plan", 2000)
    tr.track(_map(2001), start, *_frame())  # more than double the tuned size: re-tuned
    assert tr.tunes == 2 and ("autotune", 2001, True, 3) in tr.R.log


def test_tracker_without_tuning_never_tunes(fake):
    tr = slam.Tracker(CAM, 5, device="cpu")
    start = torch.tensor([1.0, 0, 0, 0, 0, 0, 0], dtype=torch.float64)
    for n in (100, 1000, 10000):
        tr.track(_map(n), start, *_frame())
    assert tr.tunes == 0 and all(e[0] == "plan" for e in tr.R.log)


def test_tracker_replans_on_capacity_overflow(fake):
    tr = slam.Tracker(CAM, 5, device="cpu", margin=1.5)
    start = torch.tensor([1.0, 0, 0, 0, 0, 0, 0], dtype=torch.float64)
    fake.extend([(gs.GS_ERR_CAPACITY, 5000), (0, 5000)])
    g = _map(10)
    pose = tr.track(g, start, *_frame())
    assert tr.replans == 1
    # the new capacity covers the pairs seen, with the margin: max(5000, 2 x 1000) x 1.5 + 1024
    assert tr.R.log[-1] == ("problem", 10, int(5000 * 1.5) + 1024)
    np.testing.assert_array_equal(pose.numpy(), start.numpy())  # the fake leaves the pose alone
    # an overflow whose count is below the old capacity still doubles it
    fake.extend([(gs.GS_ERR_CAPACITY, 10), (0, 10)])
    tr.track(g, start, *_frame())
    assert tr.R.log[-1] == ("problem", 10, int(2 * (int(5000 * 1.5) + 1024) * 1.5) + 1024)


def test_tracker_gives_up_after_repeated_overflows(fake):
    tr = slam.Tracker(CAM, 5, device="cpu")
    start = torch.tensor([1.0, 0, 0, 0, 0, 0, 0], dtype=torch.float64)
    fake.extend([(gs.GS_ERR_CAPACITY, 10 ** 6)] * 4)
    with pytest.raises(RuntimeError, match="kept overflowing"):
        tr.track(_map(10), start, *_frame())
    fake.clear()
    fake.append((6, 0))  # GS_ERR_TIMEOUT: not a capacity problem, so it is raised
    with pytest.raises(gs.GsError):
        tr.track(_map(10), start, *_frame())


class FakeMapper(FakeRasterizer):
    """The mapping side of the fake: renders a silhouette and records the gradient calls."""

    sil_value = 1.0

    def render(self, prob, g, poses, targets=None, stream=None, images=True):
        self.log.append(("render", g.n))
        return {"sil": torch.full((CAM.height * CAM.width,), self.sil_value)}

    def sync(self, stream=None):
        return SimpleNamespace(n_pairs=0)

    def mapping_grads(self, g, cams, poses, targets, chunk=2, grads=None, probs=None, stream=None):
        self.log.append(("grads", len(cams), chunk, len(probs)))
        return {"grads": grads}


def test_slam_keyframes_window_iterations_and_removal(fake, monkeypatch):
    """slam.Slam on ten frames: keyframes at 0, 4 and 8; the first keyframe's Gaussians
    from every pixel with depth, later ones only where the silhouette is low; 5 Adam
    iterations on the first keyframe, 2 after, each over the last `window` keyframes in
    chunks; removal into the spare map after every keyframe, the two maps swapping."""
    monkeypatch.setattr(gs, "Rasterizer", FakeMapper)
    monkeypatch.setattr(gs, "load", lambda *a, **k: None)
    monkeypatch.setattr(gs, "gs_map_scratch_bytes", lambda items: 256)
    monkeypatch.setattr(gs, "_ptr", lambda t: None if t is None else t.data_ptr())  # host tensors here
    monkeypatch.setattr(gs, "gs_default_map_config", lambda: gs.gs_map_config(sil_add=0.5, opacity_min=0.005))
    steps = []

    def add(cfg, m, count, cam, pose, rgb, depth, sil, scr, nb, err, stream=None):
        take = depth.reshape(-1) > 0
        if sil is not None:
            take &= sil.reshape(-1) < cfg.sil_add
        count += int(take.sum())

    def adam(cfg, m, count, grads, step, stream=None):
        steps.append(int(step))

    def prune(cfg, src, n_src, dst, n_dst, scr, nb, stream=None):
        n_dst.fill_(int(n_src.item()) - 1)  # one Gaussian faded

    monkeypatch.setattr(gs, "gs_map_add", add)
    monkeypatch.setattr(gs, "gs_map_adam_step", adam)
    monkeypatch.setattr(gs, "gs_map_prune", prune)
    cfg = slam.SlamConfig(track_iters=3, keyframe_every=4, window=2, map_iters=2, first_map_iters=5, map_chunk=1,
                          capacity=4096, prune=True)
    S = slam.Slam(CAM, cfg, device="cpu")
    first = S.map
    P = CAM.width * CAM.height
    rgb, depth = _frame()
    depth[0, :5] = 0.0  # five pixels without a measurement
    for k in range(10):
        FakeMapper.sil_value = 0.2 if k == 8 else 1.0  # frame 8 sees new surface everywhere
        S.process(k, rgb, depth, first_pose=[1.0, 0, 0, 0, 0, 0, 0] if k == 0 else None)
    assert S.stats["keyframes"] == 3 and len(S.keyframes) == 3 and len(S.poses) == 10
    # frame 0: every pixel with depth; frame 4: none (the silhouette covers it); frame 8: all again
    assert S.stats["added"] == [P - 5, 0, P - 5]
    assert S.stats["pruned"] == [1, 1, 1] and S.n == 2 * (P - 5) - 3
    assert steps == [1, 2, 3, 4, 5, 1, 2, 1, 2]
    grads = [e for e in S.mapper.log if e[0] == "grads"]
    # the window holds at most 2 keyframes, one view per chunk
    assert [e[1] for e in grads] == [1] * 5 + [2] * 2 + [2] * 2 and all(e[3] == e[1] for e in grads)
    # three removals: the maps swapped three times
    assert S.map is not first and S.spare is first
    S.close()
