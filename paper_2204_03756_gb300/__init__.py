"""GB300-native (sm_103a) mass-transfer particle-tracking (MTPT) time step.

The hot path of Schauer et al., arXiv:2204.03756 (Sec. 3): random walk with
reflecting walls, fixed-radius pair search, Gaussian weights, symmetric
normalisation and mass exchange, all in hand-written CUDA kernels behind the C
ABI of ``include/mtpt.h``.  ``mtpt`` is the ctypes binding (same names as the
C entry points), ``workloads`` the seeded input generators.
"""
from . import build, workloads  # noqa: F401
from .mtpt import (  # noqa: F401
    MTPT_DO_TRANSFER, MTPT_DO_WALK, MTPT_FP32W, MTPT_FP64, MtptError, Params, Simulation,
)
