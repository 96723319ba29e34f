"""FP64 CPU oracle for the HISQ Dslash, the even-odd normal operator and its solvers.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's
CPU-baseline leg.  The GPU library never imports, links or runs anything here.

Parity pins: every function below is pinned in tests/test_oracle_*.py against the
free-field closed form, anti-Hermiticity, gauge covariance, dense brute force on 4^4,
the paper's operation counts (Sec. 5.1) and finite differences.
"""
from .oracle import *  # noqa: F401,F403
