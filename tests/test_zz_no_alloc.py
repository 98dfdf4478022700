"""The allocation-free Gauss-Legendre entry point, gbdlt_legpts_noalloc.

Callers that cannot allocate device memory (a fixed budget owned by their own
allocator, a latency-critical path that cannot take cudaMalloc's implicit
synchronisation, a plugin handed its buffers by a host framework) get the node
kernel without a plan: its scratch lives in a static device array in the
library.  These tests call it through the C ABI on two calls in a row (the
shared scratch keeps the previous call's contents) and check every output
against the oracle's double-double nodes, with the node tolerances of the
parity tests; they also check it against the plan-based gbdlt_legpts, and
that it makes no device allocation (the library's own allocation counter and
the device's free memory both unchanged across the calls).

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import ctypes
import gc
import functools

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
    ptrs = [None if t is None else ctypes.c_void_p(t.data_ptr()) for t in outs]
    return gb.lib().gbdlt_legpts_noalloc(N, *ptrs, ctypes.c_void_p(stream.cuda_stream))


def oracle_rows(N):
    """Every node up to N = 4096, else both ends and evenly spread interior rows."""
    if N <= 4096:
        return np.arange(N)
    return np.unique(np.r_[0:16, N - 16:N, np.linspace(0, N - 1, 64).astype(np.int64)])


@functools.lru_cache(maxsize=None)
def oracle_nodes(N):
    import oracle
    return oracle.legpts(N, oracle_rows(N))


def check_vs_oracle(N, got, with_dtheta=True):
    nd = oracle_nodes(N)
    rows = oracle_rows(N)
    x, th, w = [t.cpu().numpy()[rows] for t in got[:3]]
    assert np.max(np.abs(x - nd.x)) <= 4e-16
    assert np.max(np.abs(th - nd.theta)) <= 1e-15
    assert np.max(np.abs(w - nd.w) / nd.w) <= 1e-14
    if with_dtheta:
        dth = got[3].cpu().numpy()[rows]
        assert np.max(np.abs(dth - nd["dtheta"])) * N <= 2e-14


# powers of two, odd N with a middle node, N just above 64 (where the end-node
# kernel starts), lengths that are not powers of two, and the largest N
SIZES = [1, 2, 3, 64, 65, 777, 1000, 1024, 4096, 65535, 65536]


@pytest.mark.parametrize("N", SIZES)
def test_noalloc_matches_oracle_twice(gb, N):
    stream = torch.cuda.current_stream()
    outs = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4)]
    keep = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4)]
    # one call first: the first call on a device may load the library's device
    # code (and with it the scratch array) into the context
    assert noalloc(gb, 1, [t[:1] for t in outs], stream) == 0
    # the window's own operations once before it (their first use may load device
    # code, which takes device memory)
    for t in outs:
        t.fill_(float("nan"))
    assert noalloc(gb, N, outs, stream) == 0
    check_vs_oracle(N, outs)
    for a, b in zip(keep, outs):
        a.copy_(b)
    torch.cuda.synchronize()
    # plans of earlier tests that the collector frees inside the measured window
    # would change the device's free memory: collect them first, pause collection
    gc.collect()
    gc.disable()
    try:
        allocs = gb.device_alloc_count()
        free0 = torch.cuda.mem_get_info()[0]
        for i in range(2):
            for t in outs:
                t.fill_(float("nan"))
            assert noalloc(gb, N, outs, stream) == 0
            check_vs_oracle(N, outs)
            if i == 0:
                for a, b in zip(keep, outs):
                    a.copy_(b)
        torch.cuda.synchronize()
        assert gb.device_alloc_count() == allocs
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        gc.enable()
    for a, b in zip(keep, outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("N", [3, 65, 1000, 65535])
def test_noalloc_matches_plan(gb, N):
    """The plan path on the same length (the direct method's plan for lengths
    that are not powers of two): the same node kernels, so bitwise equal."""
    stream = torch.cuda.current_stream()
    ref = gb.Plan(N).legpts()
    outs = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4)]
    assert noalloc(gb, N, outs, stream) == 0
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)


def test_noalloc_shrinking_size(gb):
    """A smaller call after a larger one: stale scratch beyond N is never read."""
    stream = torch.cuda.current_stream()
    big = [torch.empty(4096, dtype=torch.float64, device="cuda") for _ in range(4)]
    small = [torch.empty(256, dtype=torch.float64, device="cuda") for _ in range(4)]
    assert noalloc(gb, 4096, big, stream) == 0
    assert noalloc(gb, 256, small, stream) == 0
    check_vs_oracle(256, small)


def test_noalloc_without_dtheta(gb):
    stream = torch.cuda.current_stream()
    N = 512
    outs = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    assert noalloc(gb, N, outs + [None], stream) == 0
    check_vs_oracle(N, outs, with_dtheta=False)


def test_noalloc_on_side_stream(gb):
    s = torch.cuda.Stream()
    N = 2048
    outs = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(4)]
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        assert noalloc(gb, N, outs, s) == 0
    check_vs_oracle(N, outs)


def test_noalloc_rejects_bad_sizes(gb):
    stream = torch.cuda.current_stream()
    outs = [torch.empty(8, dtype=torch.float64, device="cuda") for _ in range(4)]
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in outs]
    L = gb.lib()
    s = ctypes.c_void_p(stream.cuda_stream)
    assert L.gbdlt_legpts_noalloc(65537, *ptrs, s) == -2
    assert L.gbdlt_legpts_noalloc(0, *ptrs, s) == -2
    assert L.gbdlt_legpts_noalloc(-5, *ptrs, s) == -2
    assert L.gbdlt_legpts_noalloc(8, None, ptrs[1], ptrs[2], ptrs[3], s) == -1
    assert L.gbdlt_legpts_noalloc(8, ptrs[0], None, ptrs[2], ptrs[3], s) == -1
    assert L.gbdlt_legpts_noalloc(8, ptrs[0], ptrs[1], None, ptrs[3], s) == -1
