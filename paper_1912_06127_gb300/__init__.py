"""GB300-native parallel two-site TDVP (arXiv:1912.06127) for long-range spin chains.

The compute path lives in libtdvp.so (hand-written CUDA for sm_103a behind the
C ABI of include/tdvp.h); `tdvp` is its thin ctypes binding.
"""
from . import tdvp  # noqa: F401

__all__ = ["tdvp"]
