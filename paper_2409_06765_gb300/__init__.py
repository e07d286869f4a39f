"""GB300 (sm_103a) differentiable tile-based Gaussian rasterizer (arXiv 2409.06765).

The compute path is the C-ABI library libgs.so (include/gs.h, sources in csrc/),
loaded through ``_lib`` (ctypes).  ``raster`` adds the autograd wrapper and the
paper-style ``rasterization`` call; ``synth`` draws seeded synthetic inputs.
Importing the package does not load the CUDA library; the first call does, and it
raises if libgs.so is missing or no CUDA device is present.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "raster", "_lib"]


def __getattr__(name):
    if name in ("raster", "_lib", "pipeline", "serve", "autotune", "scene_io"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
