"""The benchmark's reference arm (the FP64 oracle on the host cores) on the CPU: with more
steps than the frame has bands, every step's band stays inside the frame and the oracle's
tracking iteration runs on it (a band that ran past the bottom edge once made the arm fail
after seven steps of 64 rows on a 480-row frame)."""
import numpy as np

import bench
from paper_2408_05635_gb300 import scenes


def test_reference_steps_wrap_inside_the_frame():
    g, cam = scenes.cube_scene(n=300, seed=0)
    cam = scenes.Cam(70.0, 70.0, 39.5, 29.5, 80, 60)  # 60 rows: three 16-row bands, then a remainder
    rng = np.random.default_rng(0)
    start = scenes.perturb_pose(scenes.identity_pose(), rng, 1.0, 0.02)
    rgb = rng.uniform(size=(3, cam.height, cam.width))
    depth = rng.uniform(1.0, 3.0, size=(cam.height, cam.width))
    prior = depth.copy()
    times, cores = bench.reference_steps(g, cam, start, rgb, depth, prior, steps=9, warmup=3, band=16)
    assert len(times) == 9 and all(t > 0 for t in times)
    assert cores >= 1
