"""GPU parity at large N and for every operator of both forms.

* 4096 seeded rows at N = 2^20 and 2^22: the FP64 and FP32 DLT of decaying and
  non-decaying coefficients against the oracle's double-double row sums, and
  the IDLT's forward residual (the exact inverse satisfies
  sum_n c_n P_n(x_k) = f_k, Eq. 1 and Eq. 2) at the same rows.  The oracle's
  nodes and row sums there are stored in tests/golden/rows4096_N2p*.npz by
  tests/golden/make_rows4096.py, which calls only the oracle.
* Transposes at large N on inputs that vanish off a set of sampled rows: every
  output entry of dlt_t, chebeval_t and the IDLT is then a sum over those rows
  only, which the oracle computes exactly (Sec. 4 matrix form).
* idlt_t, leg2cheb, leg2cheb_t and chebeval at sampled output indices.
* Unit vectors at the band edges: c = e_n for n at the head block's edge, at
  every band cut +-1 and at the ends, through the DLT (f_k = P_n(x_k)); g = e_k
  for rows at every band's row range edges through dlt_t (out_n = P_n(x_k)).
  With ||c||_1 = 1 these are the sharpest checks of which band and which
  recurrence segment a column or row falls in.
* The FP32 form on every operator at N <= 4096, full vectors.
Bars (Corollary 2.2's normalisation): 1e-12 for FP64 plans, 5e-6 for FP32 plans.
"""
import functools
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 5e-6
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_00354_gb300 import build
    build.build()
    import paper_1505_00354_gb300 as g
    return g


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.double().cpu().numpy()


def tol(prec):
    return TOL64 if prec == "fp64" else TOL32


def tdtype(prec):
    return torch.float64 if prec == "fp64" else torch.float32


def gprec(gb, prec):
    return gb.FP64 if prec == "fp64" else gb.FP32


@functools.lru_cache(maxsize=None)
def golden(p2):
    """The stored oracle values at 4096 rows, after checking that the seeded
    inputs they were computed from are the ones this machine generates."""
    import oracle
    from paper_1505_00354_gb300 import inputs
    z = np.load(os.path.join(GOLDEN, f"rows4096_N2p{p2}.npz"))
    N = 2**p2
    c_flat = inputs.coeffs(N, 20 + p2, 0.0)
    c_dec = inputs.coeffs(N, 10 + p2, 1.0)
    for c, fp in ((c_flat, z["fp_flat"]), (c_dec, z["fp_dec"])):
        # the first entries bit for bit; the sums to their rounding (numpy's
        # pairwise summation may block differently on another architecture)
        assert np.array_equal(c[:8], fp[:8]), "seeded input differs from the stored one"
        assert np.allclose([c.sum(), (c * c).sum()], fp[8:], rtol=1e-9, atol=1e-6), "seeded input differs"
    nd = oracle.Nodes({k: z[k] for k in ("x_hi", "x_lo", "w_hi", "w_lo", "theta_hi", "theta_lo", "dtheta")})
    nd["k"] = z["rows"]
    nd["N"] = N
    return {"rows": z["rows"], "nodes": nd, "c_flat": c_flat, "c_dec": c_dec, "f_flat": z["f_flat"],
            "f_dec": z["f_dec"]}


def subset(nd, idx):
    """Nodes restricted to positions idx of a Nodes object."""
    import oracle
    out = oracle.Nodes({k: nd[k][idx] for k in ("x_hi", "x_lo", "w_hi", "w_lo", "theta_hi", "theta_lo", "dtheta")})
    out["k"] = nd["k"][idx]
    out["N"] = nd["N"]
    return out


@functools.lru_cache(maxsize=None)
def rows_nodes(N, count, seed):
    """Sampled rows and their oracle nodes: from the stored 4096 at 2^20 and
    2^22 (the first `count` of a fixed permutation, ends included), computed
    otherwise."""
    import oracle
    from paper_1505_00354_gb300 import inputs
    p2 = int(math.log2(N))
    if N in (2**20, 2**22):
        G = golden(p2)
        rows = G["rows"]
        ends = np.r_[0:8, rows.size - 8:rows.size]
        rest = np.setdiff1d(np.arange(rows.size), ends)
        pick = np.sort(np.r_[ends, np.random.default_rng(seed).permutation(rest)[:count - ends.size]])
        return rows[pick], subset(G["nodes"], pick)
    rows = inputs.sample_rows(N, count, seed=seed)
    return rows, oracle.legpts(N, rows)


_plans = {}


def plan(gb, N, prec):
    key = (N, prec)
    if key not in _plans:
        _plans.clear()  # one large plan at a time
        torch.cuda.empty_cache()
        _plans[key] = gb.Plan(N, gprec(gb, prec), method=gb.METHOD_FAST)
    return _plans[key]


# --------------------------------------------------------------------------
# 4096 seeded rows at 2^20 and 2^22
# --------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("decay", [0.0, 1.0])
@pytest.mark.parametrize("p2", [20, 22])
def test_dlt_rows4096(gb, p2, decay, prec):
    G = golden(p2)
    c = G["c_dec"] if decay else G["c_flat"]
    ref = G["f_dec"] if decay else G["f_flat"]
    got = host(plan(gb, 2**p2, prec).dlt(dev(c, tdtype(prec))))[G["rows"]]
    err = np.max(np.abs(got - ref)) / np.abs(c).sum()
    print(f"N=2^{p2} {prec} decay={decay}: dlt max err / ||c||_1 over {ref.size} rows = {err:.2e}")
    assert err <= tol(prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("p2", [20, 22])
def test_idlt_residual_rows4096(gb, p2, prec):
    """The IDLT's forward residual sum_n c_n P_n(x_k) - f_k at the 4096 rows
    (FP32 plans: at 1024 of them), normalised by ||c||_1."""
    import oracle
    from paper_1505_00354_gb300 import inputs
    N = 2**p2
    f = inputs.values(N, 30 + p2)
    if prec == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    c = host(plan(gb, N, prec).idlt(dev(f, tdtype(prec))))
    rows, nd = rows_nodes(N, 4096 if prec == "fp64" else 1024, 11)
    resid = oracle.dlt_rows(c, nd) - f[rows]
    err = np.max(np.abs(resid)) / np.abs(c).sum()
    print(f"N=2^{p2} {prec}: idlt forward residual / ||c||_1 over {rows.size} rows = {err:.2e}")
    assert err <= tol(prec)


# --------------------------------------------------------------------------
# every operator at large N (sparse inputs for the transposes, sampled outputs
# for the others)
# --------------------------------------------------------------------------
LARGE_N = [2**16, 2**20, 2**22]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", LARGE_N)
def test_transposes_sparse_input(gb, N, prec):
    """dlt_t, chebeval_t and the IDLT of an input supported on 192 sampled rows:
    every output entry against the oracle's sums over those rows."""
    import oracle
    rows, nd = rows_nodes(N, 192, 21)
    r = np.random.default_rng(N + 7)
    vals = r.standard_normal(rows.size)
    if prec == "fp32":
        vals = vals.astype(np.float32).astype(np.float64)
    g = np.zeros(N)
    g[rows] = vals
    p = plan(gb, N, prec)
    x = dev(g, tdtype(prec))
    s1 = np.abs(vals).sum()
    e1 = np.max(np.abs(host(p.dlt_t(x)) - oracle.dlt_t_rows(vals, nd, N))) / s1
    e2 = np.max(np.abs(host(p.chebeval_t(x)) - oracle.ndct_t_rows(vals, nd, N))) / s1
    ci = oracle.idlt_rows(vals, nd, N)
    scale = (np.arange(N) + 0.5) * np.abs(nd.w * vals).sum()
    e3 = np.max(np.abs(host(p.idlt(x)) - ci) / scale)
    print(f"N={N} {prec}: dlt_t {e1:.2e} chebeval_t {e2:.2e} idlt {e3:.2e} (input on {rows.size} rows)")
    for e in (e1, e2, e3):
        assert e <= tol(prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", LARGE_N)
def test_forward_operators_sampled(gb, N, prec):
    """idlt_t and chebeval at 256 sampled rows, leg2cheb and leg2cheb_t at 256
    sampled indices, all on dense seeded inputs."""
    import oracle
    from paper_1505_00354_gb300 import inputs
    rows, nd = rows_nodes(N, 256, 31)
    p = plan(gb, N, prec)
    y = inputs.coeffs(N, 900 + N % 1000, 1.0)
    if prec == "fp32":
        y = y.astype(np.float32).astype(np.float64)
    x = dev(y, tdtype(prec))
    sy = (np.arange(N) + 0.5) * y
    ref4 = nd.w * oracle.dlt_rows(sy, nd)
    e4 = np.max(np.abs(host(p.idlt_t(x))[rows] - ref4)) / np.abs(sy).sum()
    e5 = np.max(np.abs(host(p.chebeval(x))[rows] - oracle.ndct_rows(y, nd))) / np.abs(y).sum()
    ks = np.unique(np.r_[0:8, N - 8:N, np.random.default_rng(N).choice(N, 240, replace=False)])
    e6 = np.max(np.abs(host(p.leg2cheb(x))[ks] - oracle.leg2cheb_rows(y, ks))) / np.abs(y).sum()
    e7 = np.max(np.abs(host(p.leg2cheb_t(x))[ks] - oracle.leg2cheb_t_rows(y, ks))) / np.abs(y).sum()
    print(f"N={N} {prec}: idlt_t {e4:.2e} chebeval {e5:.2e} leg2cheb {e6:.2e} leg2cheb_t {e7:.2e}")
    for e in (e4, e5, e6, e7):
        assert e <= tol(prec)


# --------------------------------------------------------------------------
# unit vectors at the band edges
# --------------------------------------------------------------------------
def edge_columns(q, N):
    cols = {0, 1, 2, N - 2, N - 1}
    h = q["head"]
    if h:
        cols |= {h - 2, h - 1, h, h + 1}
    for ns, _, _ in q["bands"]:
        cols |= {ns - 1, ns, ns + 1}
    return sorted(c for c in cols if 0 <= c < N)


def edge_rows(q, N):
    rws = {0, 1, N // 2 - 1, N // 2, N - 2, N - 1}
    for _, ka, kb in q["bands"]:
        for k in (ka - 1, ka, kb - 1, kb):
            rws |= {k, N - 1 - k}
    return sorted(k for k in rws if 0 <= k < N)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [2**16, 2**20])
def test_dlt_unit_vectors_band_edges(gb, N, prec):
    """c = e_n for n at the head block's edge, at every band cut +-1 and at the
    ends (one batched call): f_k = P_n(x_k) at 256 sampled rows, absolute."""
    import oracle
    p = plan(gb, N, prec)
    cols = edge_columns(p.params(), N)
    C = np.zeros((len(cols), N))
    for i, n in enumerate(cols):
        C[i, n] = 1.0
    F = host(p.dlt(dev(C, tdtype(prec))))
    rows, nd = rows_nodes(N, 256, 41)
    worst = 0.0
    for i, n in enumerate(cols):
        e = np.max(np.abs(F[i, rows] - oracle.legendre_p_at(n, nd)))
        worst = max(worst, e)
        assert e <= tol(prec), (n, e)
    print(f"N={N} {prec}: columns {cols}: max |f - P_n(x_k)| = {worst:.2e}")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [2**16, 2**20])
def test_dlt_t_unit_vectors_band_edges(gb, N, prec):
    """g = e_k for rows at every band's row range edges, the middle and the ends
    (one batched call): (P^T e_k)_n = P_n(x_k) for every n, absolute."""
    import oracle
    p = plan(gb, N, prec)
    rws = edge_rows(p.params(), N)
    G = np.zeros((len(rws), N))
    for i, k in enumerate(rws):
        G[i, k] = 1.0
    out = host(p.dlt_t(dev(G, tdtype(prec))))
    nd = oracle.legpts(N, np.array(rws, dtype=np.int64))
    worst = 0.0
    for i, k in enumerate(rws):
        ref = oracle.dlt_t_rows([1.0], subset(nd, [i]), N)
        e = np.max(np.abs(out[i] - ref))
        worst = max(worst, e)
        assert e <= tol(prec), (k, e)
    print(f"N={N} {prec}: rows {rws}: max |out - P_n(x_k)| = {worst:.2e}")


# --------------------------------------------------------------------------
# FP32 form, every operator, full vectors
# --------------------------------------------------------------------------
def _idlt_err(got, ref, w, f):
    scale = (np.arange(f.size) + 0.5) * np.abs(w * f).sum()
    return np.max(np.abs(got - ref) / scale)


@pytest.mark.parametrize("N", [2, 8, 64, 512, 1024, 4096])
def test_fp32_every_operator_full(gb, N):
    import oracle
    from paper_1505_00354_gb300 import inputs
    nd = oracle.legpts(N)
    p = gb.Plan(N, gb.FP32, method=gb.METHOD_FAST)
    a = inputs.coeffs(N, 70 + N % 97, 1.0).astype(np.float32).astype(np.float64)
    b = inputs.values(N, 71 + N % 97).astype(np.float32).astype(np.float64)
    x, y = dev(a, torch.float32), dev(b, torch.float32)
    sa, sb = np.abs(a).sum(), np.abs(b).sum()
    sab = (np.arange(N) + 0.5) * a
    errs = {
        "dlt": np.max(np.abs(host(p.dlt(x)) - oracle.dlt_rows(a, nd))) / sa,
        "idlt": _idlt_err(host(p.idlt(y)), oracle.idlt(b, nd), nd.w, b),
        "dlt_t": np.max(np.abs(host(p.dlt_t(y)) - oracle.dlt_t(b, nd))) / sb,
        "idlt_t": np.max(np.abs(host(p.idlt_t(x)) - nd.w * oracle.dlt_rows(sab, nd))) / np.abs(sab).sum(),
        "leg2cheb": np.max(np.abs(host(p.leg2cheb(x)) - oracle.leg2cheb(a))) / sa,
        "leg2cheb_t": np.max(np.abs(host(p.leg2cheb_t(y)) - oracle.leg2cheb_t(b))) / sb,
        "chebeval": np.max(np.abs(host(p.chebeval(x)) - oracle.ndct_rows(a, nd))) / sa,
        "chebeval_t": np.max(np.abs(host(p.chebeval_t(y)) - oracle.ndct_t(b, nd))) / sb,
    }
    print(f"N={N} fp32: " + " ".join(f"{k} {v:.1e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v <= TOL32, k


@pytest.mark.parametrize("N", [4096, 2**16])
def test_fp32_adjoint_identities(gb, N):
    """<A y, z> = <y, A^T z> for every operator pair of an FP32 plan, to the
    FP32 form's bar."""
    from paper_1505_00354_gb300 import inputs
    p = gb.Plan(N, gb.FP32, method=gb.METHOD_FAST)
    y = dev(inputs.coeffs(N, 7), torch.float32)
    z = dev(inputs.coeffs(N, 8), torch.float32)
    for fwd, tr in ((p.dlt, p.dlt_t), (p.chebeval, p.chebeval_t), (p.leg2cheb, p.leg2cheb_t),
                    (p.idlt, p.idlt_t)):
        a = float(torch.dot(fwd(y).double(), z.double()))
        b = float(torch.dot(y.double(), tr(z).double()))
        scale = float(torch.linalg.vector_norm(y.double(), 1) * torch.linalg.vector_norm(z.double(), 1))
        assert abs(a - b) <= TOL32 * scale, (fwd.__name__, a, b)
