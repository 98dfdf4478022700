"""The FFT-based chain for N that is not a power of two (GBDLT_METHOD_FAST):
the chain runs on the next power-of-two grid G, the coefficients zero-padded to
G and the rows of the N-point Gauss-Legendre rule each expanded about their
nearest grid point (Taylor step of Sec. 2 with the bound of Corollary 2.4 taken
at |n dtheta| <= (N-1) pi / (2G)).

Every operator is compared with the oracle on full vectors up to N = 4095, odd
N included (the middle node x = 0), both forms.  Above the direct method's limit
(N = 10^5, 10^6 and 2^20 - 1) the DLT is compared at sampled rows and the IDLT
through its forward residual.  The fast and direct methods agree where both
exist; adjoint identities, batched = single bitwise, input-scale invariance
and the uneven batch with unrounded lengths complete it.  Bars as in
test_gpu_parity: 1e-12 (FP64) and 5e-6 (FP32) in the normalisations of
Corollary 2.2.
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


FULL = [3, 5, 6, 7, 100, 257, 1000, 1025, 1536, 3001, 4095]


@pytest.mark.parametrize("N", FULL)
@pytest.mark.parametrize("prec", [0, 1])
def test_grid_all_ops_full(gb, N, prec):
    import oracle
    from paper_1505_00354_gb300 import inputs
    tol, dt = (TOL64, torch.float64) if prec == 0 else (TOL32, torch.float32)
    p = gb.Plan(N, prec, method=gb.METHOD_FAST)
    q = p.params()
    assert q["method"] == gb.METHOD_FAST and q["grid_n"] == 1 << (N - 1).bit_length()
    nd = onodes(N)

    def cast(a):
        return a.astype(np.float32).astype(np.float64) if prec == 1 else a

    c = cast(inputs.coeffs(N, 1300 + N, 0.0 if N % 2 else 1.0))
    g = cast(inputs.values(N, 1400 + N))
    cn, gn = np.abs(c).sum(), np.abs(g).sum()
    s = np.arange(N) + 0.5
    errs = {}
    errs["dlt"] = np.max(np.abs(host(p.dlt(dev(c, dt))) - oracle.dlt_rows(c, nd))) / cn
    errs["chebeval"] = np.max(np.abs(host(p.chebeval(dev(c, dt))) - oracle.ndct_rows(c, nd))) / cn
    errs["leg2cheb"] = np.max(np.abs(host(p.leg2cheb(dev(c, dt))) - oracle.leg2cheb(c))) / cn
    errs["dlt_t"] = np.max(np.abs(host(p.dlt_t(dev(g, dt))) - oracle.dlt_t(g, nd))) / gn
    errs["chebeval_t"] = np.max(np.abs(host(p.chebeval_t(dev(g, dt))) - oracle.ndct_t(g, nd))) / gn
    errs["leg2cheb_t"] = np.max(np.abs(host(p.leg2cheb_t(dev(g, dt))) - oracle.leg2cheb_t(g))) / gn
    errs["idlt"] = np.max(np.abs(host(p.idlt(dev(g, dt))) - oracle.idlt(g, nd)) / (s * np.abs(nd.w * g).sum()))
    ref = nd.w * oracle.dlt_rows(s * g, nd)
    errs["idlt_t"] = np.max(np.abs(host(p.idlt_t(dev(g, dt))) - ref) / nd.w) / np.abs(s * g).sum()
    print(f"N={N} prec={prec} L={q['L']}", {k: f"{v:.1e}" for k, v in errs.items()})
    for k, e in errs.items():
        assert e <= tol, (k, e)


@pytest.mark.parametrize("N", [10**5, 10**6, 2**20 - 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_grid_sampled_rows(gb, N, prec):
    """Beyond the direct method's limit: the DLT at sampled nodes (both ends and
    uniform rows) and the IDLT through its forward residual."""
    import oracle
    from paper_1505_00354_gb300 import inputs
    tol, dt = (TOL64, torch.float64) if prec == 0 else (TOL32, torch.float32)
    p = gb.Plan(N, prec, method=gb.METHOD_FAST)
    c = inputs.coeffs(N, 1500 + N % 1000, 1.0)
    if prec == 1:
        c = c.astype(np.float32).astype(np.float64)
    rows = tuple(sorted(set(inputs.sample_rows(N, 40, 1600 + N % 1000, include_ends=8).tolist())))
    nd = onodes(N, rows)
    f = host(p.dlt(dev(c, dt)))
    e = np.max(np.abs(f[list(rows)] - oracle.dlt_rows(c, nd))) / np.abs(c).sum()
    print(f"N={N} prec={prec} grid DLT sampled error {e:.2e}")
    assert e <= tol
    # the IDLT of random values: its forward residual sum_n c_n P_n(x_k) - f_k
    # at the sampled rows, normalised by ||c||_1 (as for powers of two)
    fv = inputs.values(N, 1800 + N % 1000)
    if prec == 1:
        fv = fv.astype(np.float32).astype(np.float64)
    cb = host(p.idlt(dev(fv, dt)))
    r = oracle.dlt_rows(cb, nd) - fv[list(rows)]
    e = np.max(np.abs(r)) / np.abs(cb).sum()
    print(f"N={N} prec={prec} grid IDLT forward residual {e:.2e}")
    assert e <= tol


@pytest.mark.parametrize("N", [300, 1000, 12345, 65535])
def test_grid_matches_direct(gb, N):
    from paper_1505_00354_gb300 import inputs
    c = dev(np.stack([inputs.coeffs(N, 1700 + i, 1.0) for i in range(3)]))
    pd = gb.Plan(N, method=gb.METHOD_DIRECT)
    pf = gb.Plan(N, method=gb.METHOD_FAST)
    for op in ("dlt", "dlt_t", "idlt", "idlt_t"):
        a, b = host(getattr(pd, op)(c)), host(getattr(pf, op)(c))
        e = np.max(np.abs(a - b)) / np.abs(host(c)).sum(axis=1).max()
        assert e <= 2 * TOL64, (op, e)


@pytest.mark.parametrize("N", [1000, 3 * 2**16 + 1])
def test_grid_adjoints_batch_scale(gb, N):
    """<A y, z> = <y, A^T z> for every operator pair; batched calls equal single
    calls bitwise; scaling the input by 2^(+-700) scales the outputs exactly."""
    import paper_1505_00354_gb300.inputs as inp
    p = gb.Plan(N, method=gb.METHOD_FAST)
    y, z = dev(inp.coeffs(N, 7)), dev(inp.coeffs(N, 8))
    for fwd, tr in ((p.dlt, p.dlt_t), (p.chebeval, p.chebeval_t), (p.leg2cheb, p.leg2cheb_t),
                    (p.idlt, p.idlt_t)):
        a = float(torch.dot(fwd(y), z))
        b = float(torch.dot(y, tr(z)))
        scale = float(torch.linalg.vector_norm(y, 1) * torch.linalg.vector_norm(z, 1))
        assert abs(a - b) <= 1e-13 * scale, (fwd.__name__, a, b)
    C = dev(np.stack([inp.coeffs(N, 60 + i, 1.0) for i in range(5)]))
    for op in (p.dlt, p.idlt, p.dlt_t, p.idlt_t, p.leg2cheb, p.leg2cheb_t, p.chebeval, p.chebeval_t):
        full = op(C)
        for i in (0, 4):
            assert torch.equal(full[i], op(C[i].clone())), (op.__name__, i)
    for op in (p.dlt, p.idlt, p.dlt_t, p.idlt_t, p.leg2cheb, p.leg2cheb_t):
        yref = op(C[1].clone())
        ref = float(torch.max(torch.abs(yref)))
        for k in (-700, 700):
            ys = op(C[1] * 2.0**k) * 2.0**-k
            assert float(torch.max(torch.abs(ys - yref))) <= 1e-14 * ref, (op.__name__, k)


def test_grid_uneven_batch(gb):
    """Unrounded lengths 16 .. 8192 (log-uniform): the lengths in (G/2, G] of one
    direction share one grid group above G = 512; replays are deterministic;
    every transform matches the single plan of its own length, and a seeded
    sample matches the oracle."""
    import oracle
    from paper_1505_00354_gb300 import inputs
    rng = np.random.default_rng(44)
    B = 160
    Ns = np.round(2 ** rng.uniform(4, 13, B)).astype(np.int64)
    dirs = rng.integers(0, 2, B).astype(np.int32)
    x = np.concatenate([inputs.coeffs(int(N), 7000 + i, 1.0) for i, N in enumerate(Ns)])
    b = gb.Batch(Ns, dirs, gb.FP64)
    groups = b.groups()
    # one group per (G, direction) bucket: grid groups above 512, direct groups
    # per length below (and single-length buckets as they stand)
    assert any(G["lengths"] > 1 for G in groups)
    for G in groups:
        if G["lengths"] > 1:
            assert G["N"] > 512 and G["method"] == gb.METHOD_FAST
    assert sum(1 for G in groups if G["N"] > 512) <= 2 * 5
    xd = dev(x)
    y = b.run(xd)
    assert torch.equal(y, b.run(xd))
    check_groups(gb, b, Ns, dirs, xd, y, 0, TOL64)
    off = b.offsets
    worst = 0.0
    for i in rng.choice(B, 12, replace=False):
        N = int(Ns[i])
        xi, yi = host(xd[off[i]:off[i + 1]]), host(y[off[i]:off[i + 1]])
        nd = onodes(N)
        if dirs[i] == 0:
            err = np.max(np.abs(yi - oracle.dlt_rows(xi, nd))) / np.abs(xi).sum()
        else:
            err = np.max(np.abs(yi - oracle.idlt(xi, nd)) / ((np.arange(N) + 0.5) * np.abs(nd.w * xi).sum()))
        worst = max(worst, err)
    assert worst <= TOL64


@pytest.mark.parametrize("prec", [0, 1])
def test_grid_group_many_passes(gb, prec):
    """A grid group larger than one workspace pass (lengths 4097 .. 8192, 300
    transforms per direction: several passes of the G = 8192 chain), so the
    per-item rule table is read at every pass's offset; every transform matches
    the single plan of its own length."""
    from paper_1505_00354_gb300 import inputs
    rng = np.random.default_rng(45)
    B = 600
    Ns = rng.integers(4097, 8193, B).astype(np.int64)
    dirs = np.r_[np.zeros(B // 2), np.ones(B - B // 2)].astype(np.int32)
    x = np.concatenate([inputs.coeffs(int(N), 7500 + i, 1.0) for i, N in enumerate(Ns)])
    b = gb.Batch(Ns, dirs, prec)
    groups = b.groups()
    assert len(groups) == 2 and all(G["N"] == 8192 and G["count"] == 300 for G in groups)
    dt = torch.float64 if prec == 0 else torch.float32
    xd = dev(x, dt)
    y = b.run(xd)
    check_groups(gb, b, Ns, dirs, xd, y, prec, TOL64 if prec == 0 else TOL32)
