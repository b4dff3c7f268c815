"""GB300 (sm_103a) implementation of the COBS query path (arXiv:1905.09624).

The compute path lives in the CUDA library libcobs_gpu.so (csrc/, C ABI in
include/cobs_gpu.h); `cobs` is its thin ctypes binding.
"""
from . import cobs  # noqa: F401
from ._build import build  # noqa: F401
