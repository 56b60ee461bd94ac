"""GB300-native pseudo-spectral Navier-Stokes RK4 solver (arXiv 1602.03638).

The compute path is the CUDA library built from csrc/ (C ABI in
include/dns.h); ``Solver`` is a thin marshalling layer over it. Nothing here
computes the method on the CPU: without the built library every call raises.
"""

from .solver import Ensemble, Solver, set_tune_cache, tune_cache_lookup  # noqa: F401

__all__ = ["Solver", "Ensemble", "set_tune_cache", "tune_cache_lookup"]
