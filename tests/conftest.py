"""Shared test fixtures.  Tests marked ``gpu`` need a GB300 and the built CUDA library;
everything else runs on the CPU (the oracle, host logic, the C-ABI symbol table)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def oracle_scene(g):
    """float32 Gaussians (scenes.Gaussians) -> the oracle's FP64 copy of the same values."""
    import oracle
    return oracle.Scene(*g.arrays())


def oracle_cam(cam):
    import oracle
    return oracle.camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height)


@pytest.fixture
def rng():
    return np.random.default_rng(1234)
