"""Write the oracle's values at 4096 seeded rows for N = 2^20 and 2^22.

Calls only the CPU oracle (oracle/) and the seeded input generators; nothing
here touches the GPU library.  For each N it stores, in rows4096_N2p<p>.npz:
  rows           the 4096 sampled node indices (16 at the ends, the rest
                 uniform; seed 1000 + p)
  x_hi, x_lo, w_hi, w_lo, theta_hi, theta_lo, dtheta
                 the double-double Gauss-Legendre nodes and weights there
                 (Newton on the three-term recurrence, Eq. 1 / Sec. 2.2)
  f_flat, f_dec  Eq. 1 at those rows for c = inputs.coeffs(N, 20 + p, 0) and
                 c = inputs.coeffs(N, 10 + p, 1) (the non-decaying and
                 (n+1)^-1-decaying coefficient vectors)
  fp_flat, fp_dec
                 fingerprints of those two inputs (first 8 entries, sum, sum
                 of squares), which the tests compare before trusting f_*
Run from the repository root: python tests/golden/make_rows4096.py
(about 10 minutes on 8 cores).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1505_00354_gb300 import inputs  # noqa: E402

NROWS = 4096


def fingerprint(c):
    return np.r_[c[:8], c.sum(), (c * c).sum()]


def path(p2):
    return os.path.join(HERE, f"rows4096_N2p{p2}.npz")


def make(p2):
    N = 2**p2
    t0 = time.time()
    rows = inputs.sample_rows(N, NROWS, seed=1000 + p2)
    nd = oracle.legpts(N, rows)
    c_flat = inputs.coeffs(N, 20 + p2, 0.0)
    c_dec = inputs.coeffs(N, 10 + p2, 1.0)
    out = {"rows": rows, "f_flat": oracle.dlt_rows(c_flat, nd), "f_dec": oracle.dlt_rows(c_dec, nd),
           "fp_flat": fingerprint(c_flat), "fp_dec": fingerprint(c_dec)}
    for k in ("x_hi", "x_lo", "w_hi", "w_lo", "theta_hi", "theta_lo", "dtheta"):
        out[k] = nd[k]
    np.savez_compressed(path(p2), **out)
    print(f"N=2^{p2}: {rows.size} rows in {time.time() - t0:.0f} s -> {path(p2)}")


if __name__ == "__main__":
    for p2 in (int(a) for a in (sys.argv[1:] or ["20", "22"])):
        make(p2)
