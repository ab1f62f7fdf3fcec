"""GB300-native hot path of the adaptive domain decomposition FE/FD method
for the stabilized Maxwell system in conductive media (arXiv 2508.07780):
forward and adjoint explicit time stepping and the Lagrangian gradient with
respect to epsilon and sigma, in hand-written sm_103a CUDA behind the C ABI of
include/ddfd.h.  This package holds the ctypes binding and the build script.
"""
from .binding import (  # noqa: F401
    ABI_SYMBOLS,
    DDFDError,
    Batch,
    Problem,
    ddfd_config,
    ddfd_info,
    load_library,
    misfit_noalloc,
    LIB_PATH,
)
