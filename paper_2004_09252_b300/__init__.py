"""B300-native MemShield page cipher (arXiv 2004.09252, Sec. 4.4).

The compute path is the C-ABI CUDA library ``libmemshield.so`` (declared in
include/memshield.h, sources in csrc/); ``memshield`` is its ctypes binding.
Importing the binding loads the library and raises if it is missing.
"""
from . import build  # noqa: F401

__all__ = ["build"]
