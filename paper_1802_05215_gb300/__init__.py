"""GB300-native (sm_103a) polynomial-filtered spectrum slicing (arXiv:1802.05215).

Submodules:
  inputs  -- seeded synthetic matrices (finite-difference Laplacians, Anderson model)
  native  -- binding of the C ABI (include/evsl_gb300.h) implemented by libevsl_gb300.so
  build   -- nvcc build of libevsl_gb300.so
The native library is loaded on first use of `native`; nothing here runs on the CPU in its
place.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "native", "build"]
