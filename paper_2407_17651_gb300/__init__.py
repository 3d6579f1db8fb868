"""GB300-native PARS3: skew-symmetric SpMV with RCM reordering and a 3-way
band split, plus the MRS solver for shifted skew systems.

The CUDA library (libpars3.so, C ABI in include/pars3.h) does the work; the
``pars3`` module is its ctypes binding.  Importing this package does not load
the library; ``pars3.lib()`` does, and raises if it has not been built.
"""
from . import pars3  # noqa: F401
from .pars3 import *  # noqa: F401,F403
