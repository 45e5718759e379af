"""The seeded input generators: the torch ray-caster reproduces the numpy one, and the
long sequence's camera path moves by trackable steps."""
import numpy as np
import pytest

from paper_2408_05635_gb300 import scenes


def test_torch_raycast_matches_numpy():
    poses = scenes.spline_trajectory(50)
    cam = scenes.Cam(200.0, 200.0, 79.5, 59.5, 160, 120)
    for k in (0, 17, 33):
        a = scenes.raycast_room(poses[k], cam)
        b = scenes.raycast_room_torch(poses[k], cam)
        np.testing.assert_array_equal(a[0], b[0].numpy())
        np.testing.assert_array_equal(a[1], b[1].numpy())


def test_spline_steps_are_trackable():
    from scipy.spatial.transform import Rotation
    poses = scenes.spline_trajectory(200)
    c = np.array([-scenes.pose_rt(p)[0].T @ scenes.pose_rt(p)[1] for p in poses])
    step = np.linalg.norm(np.diff(c, axis=0), axis=1)
    ang = [np.degrees(np.linalg.norm(Rotation.from_matrix(scenes.pose_rt(a)[0] @ scenes.pose_rt(b)[0].T).as_rotvec()))
           for a, b in zip(poses[:-1], poses[1:])]
    assert step.max() < 0.1 and max(ang) < 8.0
    X, Y, Z = scenes.ROOM
    assert np.all(c[:, 0] > 0.5) and np.all(c[:, 0] < X - 0.5) and np.all(c[:, 2] > 0.5) and np.all(c[:, 2] < Z - 0.5)


def test_camera_centres_and_trajectory_report():
    """The sequence driver's camera centres and the bench's trajectory report against the
    metric oracle's independent definitions (closed forms of a shifted trajectory)."""
    import bench
    from oracle import metrics as omx
    from paper_2408_05635_gb300 import slam
    poses = np.asarray(scenes.spline_trajectory(30, seed=4))
    np.testing.assert_allclose(slam.camera_centres(poses), [omx.camera_centre(p) for p in poses], atol=1e-12)
    rep = bench._trajectory_report(poses, poses)
    assert rep["ate_rmse_cm"] == 0.0 and rep["max_rot_err_deg"] == 0.0
    shifted = []
    for p in poses:
        R, t = scenes.pose_rt(p)
        shifted.append(scenes.pose_from_rt(R, t - R @ np.array([0.0, 0.03, 0.04])))
    rep = bench._trajectory_report(np.asarray(shifted), poses)
    ref = omx.trajectory_errors(shifted, poses)
    assert rep["ate_rmse_cm"] == pytest.approx(5.0, abs=1e-6)
    assert rep["ate_rmse_cm"] == pytest.approx(100 * ref["ate_rmse"], abs=1e-6)


def test_kernel_rooflines_arithmetic():
    """The bench's per-kernel roofline table: bytes or FLOPs per launch over the event
    time, against the measured HBM bandwidth or the FP32 FMA peak (hand-computed cases)."""
    import bench
    ms = {"k_project": 0.01, "k_forward": 0.05, "k_finalize": 0.01, "k_scan_tiles": 0.01}
    r = bench.kernel_rooflines(ms, n_gauss=1000, views=2, attr_bytes=44, records=500, pairs=0,
                               fwd_contrib=10 ** 6, bwd_contrib=0, mhz=1000.0, n_sm=152)
    hbm, _ = bench.hbm_peak_gbs()
    assert r["k_project"]["achieved"] == pytest.approx((12 * 2000 + 140 * 500) / 1e-5 / 1e9, rel=1e-3)
    assert r["k_project"]["frac"] == pytest.approx(r["k_project"]["achieved"] / hbm, rel=1e-2)
    peak = 152 * 128 * 2 * 1e9 / 1e12
    assert r["k_forward"]["peak"] == pytest.approx(peak, rel=1e-3)
    assert r["k_forward"]["achieved"] == pytest.approx(23e6 / 5e-5 / 1e12, rel=1e-3)
    assert r["k_finalize"]["bound"] == "latency" and r["k_scan_tiles"] == {"bound": "latency", "us": 10.0}


def test_oracle_single_thread_small_case_rate():
    """The bench's single-thread oracle sample runs on one thread and reports a rate."""
    import bench
    import oracle
    before = oracle.num_threads(oracle.Params())
    r = bench.oracle_small_single_thread(0.2)
    assert r["cores"] == 1 and r["value"] > 0 and r["iters_per_s"] > 0
    assert oracle.num_threads(oracle.Params()) == before  # restored for whatever runs next
