"""GB300-native differentiable 3D-Gaussian rasterizer for RGB-D SLAM tracking and mapping
(arXiv 2408.05635): projection, tile binning and depth sort, front-to-back compositing
of RGB, depth and silhouette (Eqs. 2-4), the combined tracking loss, reverse
compositing to Gaussian-parameter and pose gradients, and the decoupled
rotation/translation pose update (Sec. III-B).

The compute runs in hand-written sm_103a CUDA kernels behind a C ABI (``include/gs.h``,
``csrc/``). ``gs`` is the thin ctypes binding with the same entry-point names;
``autograd`` wraps the forward/backward pair as a ``torch.autograd.Function``;
``scenes`` draws the seeded synthetic inputs.  Submodules load lazily so that
``scenes`` can be imported without the CUDA library.
"""
import importlib

__all__ = ["gs", "autograd", "scenes", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
