"""GB300 (sm_103a) implementation of the upwind-SBP velocity-stress elastic wave
scheme of Duru, Fung & Williams (arXiv 2011.02600) on curvilinear meshes.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/sbp.h``); ``_lib`` binds it with ctypes and ``solver`` manages
device buffers through PyTorch.  There is no CPU fallback.
"""
from ._lib import SbpError, lib  # noqa: F401
from .solver import ElasticSolver  # noqa: F401
