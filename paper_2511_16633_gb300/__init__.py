"""GB300-native Hessian-free ray-Born update (arXiv 2511.16633).

The compute path is librb.so (CUDA kernels for sm_103a behind the C-ABI of
include/rb.h); ``rb`` is its ctypes binding and ``recon`` a thin driver that
owns device buffers and runs frequency sweeps through the same entry points.
"""
from . import rb  # noqa: F401
