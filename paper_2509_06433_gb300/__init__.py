"""GB300 (sm_103a) differentiable tile-based 3D-Gaussian rasterizer.

The hot path of the Gaussian-splatting SLAM mapping / tracking loop: projection,
tile binning and radix sort, alpha compositing, and the backward pass to the
Gaussians and camera poses, behind the C ABI of ``include/gs.h``.
"""
from .build import build  # noqa: F401

__all__ = ["build"]


def __getattr__(name):
    # the torch-facing API is imported lazily so that building needs no GPU
    if name in ("api", "_lib"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
