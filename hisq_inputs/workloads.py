"""Workload definitions: lattice sizes, link-disorder scales, seeds, masses, tolerances.

The paper measures on production HISQ ensembles, which are not available here; these
synthetic workloads stand in for them (seeded SU(3) links U = exp(i eps H), fat = U,
long = -1/24 U U U, Gaussian sources).  Seeds: links 1000 + n, sources 2000 + 100 n + rhs,
gauge transforms 3000, uneven batch links 1100 + index.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple
    eps: float
    link_seed: int
    source_seed: int
    mass: float
    tol: float = 1e-10
    nrhs: tuple = (1,)
    shifts: tuple = ()
    compression: int = 18
    notes: str = ""


def log_shifts(n=14, lo=1e-5, hi=1.0):
    import math
    return tuple(math.exp(math.log(lo) + i * (math.log(hi) - math.log(lo)) / (n - 1)) for i in range(n))


# small FP64 case the oracle finishes in seconds
PLAIN_8x4 = Workload("plain-fp64-cg-8^4", (8, 8, 8, 8), 0.3, 1000, 2000, 0.1)
# mixed precision vs plain FP64 CG
MIXED_32x8 = Workload("mixed-cg-32^3x8", (32, 32, 32, 8), 0.5, 1001, 2100, 0.01)
# batched multi-RHS and multi-shift
BATCH_64x16 = Workload("batched-64^3x16", (64, 64, 64, 16), 0.3, 1002, 2200, 0.01,
                       nrhs=(1, 4, 8, 16), shifts=log_shifts())
# learned preconditioner
LEARNED_32x8 = Workload("learned-32^3x8", (32, 32, 32, 8), 0.5, 1003, 2300, 0.005)
# largest single-GPU lattice, 12-real compressed links
LARGE_96x24 = Workload("multishift-96^3x24", (96, 96, 96, 24), 0.3, 1004, 2400, 0.01,
                       shifts=log_shifts(), compression=12)
# side-by-side with the paper's single-device table
PAPER_32x4 = Workload("paper-32^4", (32, 32, 32, 32), 0.3, 1005, 2500, 0.01, nrhs=tuple(range(1, 13)))


def uneven_batch():
    """32 uneven lattices Ns^3 x Nt, sorted by volume (8^3x8 ... 24^3x8)."""
    dims = []
    for ns in range(8, 25, 2):
        for nt in (8, 10, 12, 16):
            if ns ** 3 * nt <= 24 ** 3 * 8:
                dims.append((ns, ns, ns, nt))
    dims += [(8, 8, 8, 24), (12, 12, 12, 24)]
    dims = sorted(set(dims), key=lambda d: (d[0] * d[1] * d[2] * d[3], d))
    return dims
