"""GB300-native (sm_103a) particle update of the unified stochastic particle
ESBGK method (USP-ESBGK, Fei, Zhang, Li, Liu, arXiv:1808.03801).

The compute path is libusp.so (hand-written CUDA kernels behind the C ABI in
include/usp.h); this package is its thin Python binding plus the synthetic
workload definitions and the serving loop.
"""
from . import workloads  # noqa: F401
from .usp import Batch, Simulation, UspError, debug_philox, lib  # noqa: F401

__all__ = ["Simulation", "Batch", "UspError", "debug_philox", "lib", "workloads"]
