"""The direct method (GBDLT_METHOD_DIRECT): the sums of Eq. (1) and (2) by the
three-term recurrence at the Legendre nodes, for any N <= 65536, and the
batch executor's per-group method choice.

Every transform is compared with the oracle's direct sums (full vectors up to
N = 4096, including lengths that are not powers of two and odd N, whose middle
node is x = 0), with sampled rows above; the direct and FFT-based methods are
compared with each other at powers of two.  Bars as in test_gpu_parity: 1e-12
(FP64) and 5e-6 (FP32) in the normalisations of Corollary 2.2.
"""
import functools

import numpy as np
import pytest
from batch_check import check_groups

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 5e-6


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_00354_gb300 import build
    build.build()
    import paper_1505_00354_gb300 as g
    return g


@functools.lru_cache(maxsize=None)
def onodes(N, rows=None):
    import oracle
    return oracle.legpts(N, None if rows is None else np.array(rows, dtype=np.int64))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.double().cpu().numpy()


FULL = [2, 3, 5, 7, 16, 33, 100, 255, 256, 257, 511, 1000, 1024, 1031, 3000, 4096]


@pytest.mark.parametrize("N", FULL)
@pytest.mark.parametrize("prec", [0, 1])
def test_direct_all_ops_full(gb, N, prec):
    import oracle
    from paper_1505_00354_gb300 import inputs
    tol, dt = (TOL64, torch.float64) if prec == 0 else (TOL32, torch.float32)
    p = gb.Plan(N, prec, method=gb.METHOD_DIRECT)
    assert p.params()["method"] == gb.METHOD_DIRECT
    nd = onodes(N)
    c = inputs.coeffs(N, 300 + N, 0.0 if N % 2 else 1.0)
    if prec == 1:
        c = c.astype(np.float32).astype(np.float64)
    cn = np.abs(c).sum()
    # DLT
    f = host(p.dlt(dev(c, dt)))
    e = np.max(np.abs(f - oracle.dlt_rows(c, nd))) / cn
    assert e <= tol, ("dlt", e)
    # DLT^T
    g = inputs.values(N, 400 + N)
    if prec == 1:
        g = g.astype(np.float32).astype(np.float64)
    got = host(p.dlt_t(dev(g, dt)))
    e = np.max(np.abs(got - oracle.dlt_t(g, nd))) / np.abs(g).sum()
    assert e <= tol, ("dlt_t", e)
    # IDLT: normalised by (n + 1/2) ||w f||_1
    got = host(p.idlt(dev(g, dt)))
    s = np.arange(N) + 0.5
    e = np.max(np.abs(got - oracle.idlt(g, nd)) / (s * np.abs(nd.w * g).sum()))
    assert e <= tol, ("idlt", e)
    # IDLT^T = D_w P D_s g
    got = host(p.idlt_t(dev(g, dt)))
    ref = nd.w * oracle.dlt_rows(s * g, nd)
    e = np.max(np.abs(got - ref) / nd.w) / np.abs(s * g).sum()
    assert e <= tol, ("idlt_t", e)


@pytest.mark.parametrize("N", [2**13, 12345, 2**16])
def test_direct_sampled_rows(gb, N):
    """Large direct plans: the DLT at sampled nodes, and the IDLT through its
    forward residual (the DLT of the computed coefficients at sampled nodes
    reproduces f, since the IDLT inverts the DLT exactly)."""
    import oracle
    from paper_1505_00354_gb300 import inputs
    p = gb.Plan(N, method=gb.METHOD_DIRECT)
    c = inputs.coeffs(N, 500 + N % 1000, 1.0)
    rows = tuple(sorted(set(inputs.sample_rows(N, 48, 600 + N % 1000).tolist())))
    nd = onodes(N, rows)
    f = host(p.dlt(dev(c)))
    e = np.max(np.abs(f[list(rows)] - oracle.dlt_rows(c, nd))) / np.abs(c).sum()
    print(f"N={N} direct DLT sampled error {e:.2e}")
    assert e <= TOL64
    cb = host(p.idlt(dev(f)))
    r = oracle.dlt_rows(cb, nd) - f[list(rows)]
    e = np.max(np.abs(r)) / np.abs(cb).sum()
    print(f"N={N} direct IDLT forward residual {e:.2e}")
    assert e <= TOL64


@pytest.mark.parametrize("N", [512, 1024, 4096])
def test_direct_matches_fast(gb, N):
    from paper_1505_00354_gb300 import inputs
    c = dev(np.stack([inputs.coeffs(N, 700 + i, 1.0) for i in range(5)]))
    pd = gb.Plan(N, method=gb.METHOD_DIRECT)
    pf = gb.Plan(N, method=gb.METHOD_FAST)
    for op in ("dlt", "dlt_t", "idlt", "idlt_t"):
        a, b = host(getattr(pd, op)(c)), host(getattr(pf, op)(c))
        e = np.max(np.abs(a - b)) / np.abs(host(c)).sum(axis=1).max()
        assert e <= 2 * TOL64, (op, e)


def test_direct_batched_bitwise(gb):
    from paper_1505_00354_gb300 import inputs
    N = 1000
    p = gb.Plan(N, method=gb.METHOD_DIRECT)
    C = dev(np.stack([inputs.coeffs(N, 800 + i, 1.0) for i in range(9)]))
    for op in ("dlt", "dlt_t", "idlt", "idlt_t"):
        full = getattr(p, op)(C)
        for i in (0, 4, 8):
            assert torch.equal(full[i], getattr(p, op)(C[i].clone())), (op, i)


@pytest.mark.parametrize("method", [0, 1, 2])
def test_batch_methods(gb, method):
    """Batches under each method choice: every transform equals the single-plan
    call of the method its group ran (bitwise; grid groups within the
    tolerance), and the autotuner's choice is the faster of its two timings."""
    from paper_1505_00354_gb300 import inputs
    rng = np.random.default_rng(90)
    Ns = (2 ** np.round(rng.uniform(4, 12, 600))).astype(np.int64)
    Ns[::7] = rng.integers(3, 3000, Ns[::7].size)  # and lengths that are not powers of two
    dirs = rng.integers(0, 2, Ns.size).astype(np.int32)
    x = np.concatenate([inputs.coeffs(int(n), 91000 + i, 1.0) for i, n in enumerate(Ns)])
    b = gb.Batch(Ns, dirs, gb.FP64, method=method)
    groups = b.groups()
    assert sum(G["lengths"] for G in groups) == len(set(zip(Ns.tolist(), dirs.tolist())))
    for G in groups:
        if method in (1, 2):
            assert G["method"] == method
        if G["lengths"] > 1:
            assert method != 2 and G["method"] == 1
        if method == 0 and G["ms_fast"] > 0 and G["ms_direct"] > 0:
            assert G["method"] == (2 if G["ms_direct"] < G["ms_fast"] else 1)
    if method == 0:  # single-length buckets are timed both ways
        assert sum(1 for G in groups if G["ms_fast"] > 0 and G["ms_direct"] > 0) >= 4
    xd = dev(x)
    y = b.run(xd)
    check_groups(gb, b, Ns, dirs, xd, y, 0, TOL64)
    print("groups:", [(G["N"], G["dir"], G["method"], round(G["ms_fast"], 3), round(G["ms_direct"], 3))
                      for G in groups][:12])
