"""GB300 (sm_103a) library for the kernel-compensated Yee-scheme Maxwell
eigenproblem in anisotropic photonic crystals (arXiv:2511.17107).

The compute path is the C ABI of ``libpcx.so`` (include/pcx.h); the module
``pcx`` is its ctypes binding.  Importing this package does not load the
library; the first call through ``pcx`` does, and raises if it is missing.
"""
from . import pcx  # noqa: F401
