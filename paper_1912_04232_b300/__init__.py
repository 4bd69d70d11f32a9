"""B300-native (sm_103a) hot path of the molecular-dynamics method of
"JAX, M.D.: A Framework for Differentiable Physics" (arXiv:1912.04232).

All hot-path work runs in the CUDA kernels of ``libjmd.so`` behind the C ABI
in ``include/jmd.h``; ``jmd`` is the thin ctypes binding with the same
names.  Importing this package fails if ``libjmd.so`` has not been built.
"""
from . import jmd  # noqa: F401
from .jmd import *  # noqa: F401,F403

__version__ = "0.1.0"
