"""The allocation-free Gauss-Legendre entry point, gbdlt_legpts_noalloc.

Callers that cannot allocate device memory (a fixed budget owned by their own
allocator, a latency-critical path that cannot take cudaMalloc's implicit
synchronisation, a plugin handed its buffers by a host framework) get the node
kernel without a plan: its scratch lives in a static device array in the
library.  These tests call it through the C ABI and compare it with the
plan-based gbdlt_legpts on two calls in a row (the shared scratch keeps the
previous call's contents), with the node tolerances of the parity tests.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_00354_gb300 import build
    build.build()
    import paper_1505_00354_gb300 as g
    return g


def noalloc(gb, N, outs, stream):
    return gb.lib().gbdlt_legpts_noalloc(N, *[ctypes.c_void_p(t.data_ptr()) for t in outs],
                                         ctypes.c_void_p(stream.cuda_stream))


def check_close(N, got, ref):
    x, th, w, dth = [t.cpu().numpy() for t in got]
    xr, thr, wr, dthr = [t.cpu().numpy() for t in ref]
    assert np.max(np.abs(x - xr)) <= 4e-16
    assert np.max(np.abs(th - thr)) <= 1e-15
    assert np.max(np.abs(w - wr) / wr) <= 1e-14
    assert np.max(np.abs(dth - dthr)) * N <= 2e-14


@pytest.mark.parametrize("N", [1, 2, 64, 1024, 65536])
def test_noalloc_matches_plan_twice(gb, N):
    stream = torch.cuda.current_stream()
    ref = gb.Plan(N).legpts()
    outs = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4)]
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(2):
        for t in outs:
            t.fill_(float("nan"))
        assert noalloc(gb, N, outs, stream) == 0
        check_close(N, outs, ref)
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before


def test_noalloc_shrinking_size(gb):
    """A smaller call after a larger one: stale scratch beyond N is never read."""
    stream = torch.cuda.current_stream()
    big = [torch.empty(4096, dtype=torch.float64, device="cuda") for _ in range(4)]
    small = [torch.empty(256, dtype=torch.float64, device="cuda") for _ in range(4)]
    assert noalloc(gb, 4096, big, stream) == 0
    assert noalloc(gb, 256, small, stream) == 0
    check_close(256, small, gb.Plan(256).legpts())


def test_noalloc_without_dtheta(gb):
    stream = torch.cuda.current_stream()
    N = 512
    outs = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    st = gb.lib().gbdlt_legpts_noalloc(N, *[ctypes.c_void_p(t.data_ptr()) for t in outs], None,
                                       ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    x, th, w, _ = gb.Plan(N).legpts()
    assert torch.equal(outs[0], x) or float((outs[0] - x).abs().max()) <= 4e-16


def test_noalloc_rejects_bad_sizes(gb):
    stream = torch.cuda.current_stream()
    outs = [torch.empty(8, dtype=torch.float64, device="cuda") for _ in range(4)]
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in outs]
    L = gb.lib()
    s = ctypes.c_void_p(stream.cuda_stream)
    assert L.gbdlt_legpts_noalloc(65537, *ptrs, s) == -2
    assert L.gbdlt_legpts_noalloc(0, *ptrs, s) == -2
    assert L.gbdlt_legpts_noalloc(8, None, ptrs[1], ptrs[2], ptrs[3], s) == -1
