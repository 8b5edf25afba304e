"""GB300 (sm_103a) differentiable omnidirectional Gaussian rasterizer (ODGS, arXiv 2410.20686).

The compute path is the C-ABI CUDA library ``libodgs.so`` (declared in ``include/odgs.h``);
``rasterizer`` marshals torch tensors into it. Importing this package does not load the
library; ``rasterizer.Rasterizer`` does, and fails loudly if it has not been built.
"""
__all__ = ["build", "scenes", "rasterizer"]


def __getattr__(name):
    if name in ("rasterizer", "scenes", "build", "_lib"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    if name in ("Rasterizer", "RenderSettings", "ODGSRender", "render"):
        from . import rasterizer
        return getattr(rasterizer, name)
    raise AttributeError(name)
