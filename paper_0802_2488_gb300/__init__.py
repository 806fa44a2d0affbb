"""GB300-native (sm_103a) implementation of the augmented-Lagrangian FFT
scheme with the discrete Green operator of Willot & Pellegrini
(arXiv:0802.2488) for 2D elastic-perfectly plastic porous lattices.

The computation lives in ``libepfft.so`` (CUDA kernels behind the C ABI of
``include/epfft.h``); :mod:`.binding` wraps it.  :mod:`.inputs` states the
synthetic workloads.  Importing this package does not need a GPU; the first
call into the library loads it and fails loudly if it is missing.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "binding", "build"]


def __getattr__(name):
    if name in ("binding", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
