"""GB300-native matrix-free Levenberg-Marquardt with residual sampling for
3D Gaussian splatting: the C-ABI library liblmrs (CUDA, sm_103a) and its
thin Python binding.

``paper_2504_12905_gb300.lmrs`` mirrors include/lmrs.h function by function;
``paper_2504_12905_gb300.synthetic`` draws seeded scenes and cameras.
"""
from . import synthetic  # noqa: F401

__all__ = ["synthetic", "lmrs", "build"]


def __getattr__(name):
    if name in ("lmrs", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
