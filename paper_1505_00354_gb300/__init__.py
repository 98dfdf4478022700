"""Fast discrete Legendre transform on one GB300 GPU.

Hale & Townsend, "A fast FFT-based discrete Legendre transform": the DLT
(Eq. 1) and IDLT (Eq. 2) computed as a Legendre -> Chebyshev conversion
(asymptotic expansion of P_n(cos theta) summed by DCT/DST over theta-bands,
recurrence elsewhere; Sec. 3) and the Taylor-series non-uniform DCT at the
Legendre nodes (Sec. 2), with the transposed chain for the IDLT (Sec. 4).
All arithmetic runs in the CUDA library built from ``csrc/``; this package
only marshals arguments to it (see ``_binding.py`` and ``include/gbdlt.h``).
"""
from ._binding import (FP32, FP64, METHOD_AUTO, METHOD_DIRECT, METHOD_FAST, Batch, GbdltError, Plan, chebeval, chebeval_t, device_alloc_count, dlt, dlt_t, fp64_fma_rate, get_plan,
                       idlt, idlt_t, launch_count, leg2cheb, leg2cheb_t, legpts, lib, plan_params)

__all__ = [
    "FP32", "FP64", "METHOD_AUTO", "METHOD_DIRECT", "METHOD_FAST", "Batch", "GbdltError", "Plan", "chebeval", "chebeval_t", "device_alloc_count", "dlt", "dlt_t", "fp64_fma_rate", "get_plan",
    "idlt", "idlt_t", "launch_count", "leg2cheb", "leg2cheb_t", "legpts", "lib", "plan_params",
]
