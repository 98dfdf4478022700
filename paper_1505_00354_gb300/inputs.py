"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU baseline.

Holds none of the method's arithmetic: only random vectors with the
distributions of the paper's experiments (Sec. 2.5, Sec. 3.1, Sec. 4.1:
normally distributed entries scaled to an algebraic decay rate) drawn from
numpy's PCG64 generator, in FP64, so that the GPU path and the oracle see the
same bits.
"""
from __future__ import annotations

import numpy as np


def coeffs(N: int, seed: int, decay: float = 0.0) -> np.ndarray:
    """c_n = z_n (n+1)^-decay, z_n ~ N(0,1) i.i.d. (decay 0: non-decaying)."""
    z = np.random.default_rng(seed).standard_normal(N)
    if decay:
        z = z * (np.arange(N, dtype=np.float64) + 1.0) ** (-decay)
    return z


def values(N: int, seed: int) -> np.ndarray:
    """f_k ~ N(0,1) i.i.d. (IDLT inputs: function values, no decay; Sec. 4.1)."""
    return np.random.default_rng(seed).standard_normal(N)


def sample_rows(N: int, count: int, seed: int, include_ends: int = 8) -> np.ndarray:
    """Sorted distinct row indices: `include_ends` rows at each end (where the
    nodes crowd and the recurrence region is longest) plus uniform random rows."""
    ends = np.r_[np.arange(min(include_ends, N)), np.arange(max(N - include_ends, 0), N)]
    count = min(count, N)
    rest = max(count - ends.size, 0)
    rng = np.random.default_rng(seed)
    pool = np.setdiff1d(np.arange(N), ends) if N <= 1 << 24 else None
    pick = rng.choice(pool, size=min(rest, pool.size), replace=False) if rest else np.array([], int)
    return np.unique(np.r_[ends, pick]).astype(np.int64)
