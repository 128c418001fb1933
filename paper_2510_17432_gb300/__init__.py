"""GB300 (sm_103a) library for the concurrent Chebyshev stochastic-propagation hot path.

The compute path is libtbpm.so (CUDA kernels behind the C ABI of include/tbpm.h);
`capi` is its thin ctypes binding with the same function names.  Importing this
package does not load the library; the first call through `capi` does, and raises
if the library has not been built (there is no CPU fallback).
"""
from . import capi  # noqa: F401
from ._build import LIB, build  # noqa: F401

__all__ = ["capi", "build", "LIB"]
