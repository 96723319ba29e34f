"""GB300 HISQ staggered Dslash and even-odd Krylov solvers (C ABI in include/hisq.h)."""
from . import hisq  # noqa: F401
from .hisq import BF16, F16, F32, F64, F64X, Context, Field, HisqError  # noqa: F401
