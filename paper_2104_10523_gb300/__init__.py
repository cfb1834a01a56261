"""GB300-native tensor-network amplitude engine (arXiv 2104.10523, Sec. 3.1).

The work runs in libtnq (C ABI, include/tnq.h): host planner in C++ and
hand-written sm_103a CUDA kernels.  ``tnq`` is the thin ctypes binding.
"""
from . import build  # noqa: F401
