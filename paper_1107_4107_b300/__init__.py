"""B300-native ensemble propagator for the Arnold-web scan of arXiv:1107.4107.

The hot path (map iteration with tangent vector, indicators, statistics,
adjoint and batched launch) runs in the CUDA library ``libarnold.so`` behind a
C ABI (``include/arnold.h``); this package is its thin ctypes binding.
Importing the package does not load the library; the first call does, and it
fails loudly when the library is missing.
"""
__all__ = ["api", "inputs", "params"]


def __getattr__(name):
    if name in ("ArnoldEnsemble", "probe_peak", "ArnoldError"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
