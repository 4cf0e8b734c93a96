"""GB300-native batched XPBD tissue simulator (FF-SRL method, arXiv 2503.18616).

The compute path is the CUDA library libffsrl.so (C ABI in include/ffsrl.h);
``ffsrl`` is its ctypes binding and ``inputs`` the seeded synthetic workloads.
The library is loaded lazily on first use and its absence is an error.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "ffsrl", "build"]
