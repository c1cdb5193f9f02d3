"""B300 VINet view interpolation (arXiv 2112.10603): Python binding of libfvv.so.

The package re-exports the C ABI (fvv_*) with the same names plus a small
Interpolator convenience class; all computation happens in libfvv.so.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import FvvError, lib, fvv_opts  # noqa: F401
from .interp import Interpolator  # noqa: F401
