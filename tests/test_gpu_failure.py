"""Failure path: a node iteration that does not settle surfaces as a status.

The Newton solve of Sec. 2.2 settles in a few iterations; the node kernels cap
it and flag a node that has not settled in a device status word, which
gbdlt_plan_sync reports as GBDLT_ERR_NOT_CONVERGED.  A plan's cap can be
lowered (gbdlt_plan_set_node_iterations), which reaches that status with no
fault, no wait and no invalid input: every loop stays bounded and the kernels
write in bounds whatever the cap.  The tests check the status, that sync clears
it, that the plan and a second plan on the same device are clean afterwards,
and that restoring the cap restores the nodes (against the oracle).
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NOT_CONVERGED = -5


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_00354_gb300 import build
    build.build()
    import paper_1505_00354_gb300 as g
    return g


@pytest.mark.parametrize("N,cap", [(48, 0), (1024, 0), (1024, 1), (1 << 16, 1)])
def test_node_iteration_cap_reports_not_converged(gb, N, cap):
    import oracle
    L = gb.lib()
    p = gb.Plan(N)
    other = gb.Plan(256)
    p.set_node_iterations(cap)
    assert L.gbdlt_legpts(p.handle, None, None, None, None) == 0  # enqueue succeeds
    assert L.gbdlt_plan_sync(p.handle) == NOT_CONVERGED
    # the status word is cleared by the sync that reported it
    assert L.gbdlt_plan_sync(p.handle) == 0
    # a second plan on the same device never saw the failure
    assert L.gbdlt_plan_sync(other.handle) == 0
    x2, _, w2, _ = other.legpts()
    other.sync()
    nd2 = oracle.legpts(256)
    assert float(np.max(np.abs(x2.cpu().numpy() - nd2.x))) <= 4e-16
    # restoring the cap restores the rule
    p.set_node_iterations(24)
    x, th, w, dth = p.legpts()
    p.sync()
    rows = np.arange(N) if N <= 4096 else np.unique(np.r_[0:8, N - 8:N, np.linspace(0, N - 1, 48).astype(int)])
    nd = oracle.legpts(N, rows)
    assert float(np.max(np.abs(x.cpu().numpy()[rows] - nd.x))) <= 4e-16
    assert float(np.max(np.abs(w.cpu().numpy()[rows] - nd.w) / nd.w)) <= 1e-14
    # transforms after the recovery run as before
    c = torch.ones(N, dtype=torch.float64, device="cuda")
    f = p.dlt(c)
    p.sync()
    assert bool(torch.isfinite(f).all())


def test_node_iteration_cap_range(gb):
    L = gb.lib()
    p = gb.Plan(64)
    for bad in (-1, 25, 1000):
        assert L.gbdlt_plan_set_node_iterations(p.handle, bad) == -1
    assert L.gbdlt_plan_set_node_iterations(None, 4) == -1
    for ok in (0, 1, 24):
        assert L.gbdlt_plan_set_node_iterations(p.handle, ok) == 0
    p.set_node_iterations(24)
    p.legpts()
    assert L.gbdlt_plan_sync(p.handle) == 0


def test_sync_reports_before_clearing_once(gb):
    """Two failing node calls before one sync: one report, then clean."""
    L = gb.lib()
    p = gb.Plan(512)
    p.set_node_iterations(0)
    for _ in range(2):
        assert L.gbdlt_legpts(p.handle, None, None, None, None) == 0
    assert L.gbdlt_plan_sync(p.handle) == NOT_CONVERGED
    assert L.gbdlt_plan_sync(p.handle) == 0
    assert ctypes.c_int(L.gbdlt_plan_sync(p.handle)).value == 0


def test_staged_copy_wait_limit_reports_error(gb):
    """A staged FFT pass whose tile-copy wait runs out (a limit of 0 cycles)
    records it: the next sync returns GBDLT_ERR_CUDA once, the context stays
    usable, and with the default limit the plan's results are again bitwise
    those of the per-thread-load passes."""
    import paper_1505_00354_gb300.inputs as inp
    L = gb.lib()
    N = 1 << 20
    p = gb.Plan(N, gb.FP32, method=gb.METHOD_FAST)
    x = torch.tensor(inp.coeffs(N, 5), dtype=torch.float32, device="cuda")
    p.set_fft_staging(False)
    ref = p.dlt(x).clone()
    p.set_fft_staging(True)
    p.set_wait_limit(0)
    p.dlt(x)
    assert L.gbdlt_plan_sync(p.handle) == -3
    assert L.gbdlt_plan_sync(p.handle) == 0
    p.set_wait_limit(1 << 32)
    y = p.dlt(x)
    assert L.gbdlt_plan_sync(p.handle) == 0
    assert torch.equal(y, ref)
    for bad in (-1, (1 << 32) + 1):
        assert L.gbdlt_plan_set_wait_limit(p.handle, bad) == -1
