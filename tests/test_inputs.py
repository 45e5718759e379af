"""The seeded input generators: the torch ray-caster reproduces the numpy one, and the
long sequence's camera path moves by trackable steps."""
import numpy as np

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
