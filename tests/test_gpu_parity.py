"""GPU parity: every entry point of the C ABI against the CPU oracle.

Inputs come from the seeded generators in paper_1505_00354_gb300.inputs (the
distributions of the paper's experiments).  Error measures:
  * DLT / NDCT / leg2cheb: max_k |f_gpu - f_oracle| / ||c||_1  (Corollary 2.2's
    normalisation); bar 1e-12 for the FP64 form, 5e-6 for the FP32 form.
  * IDLT: max_n |c_gpu - c_oracle| / ((n+1/2) ||w f||_1), the same bound carried
    through the transposed chain; same bars.
  * nodes: |x_gpu - x|, |w_gpu - w|/w, N |dtheta_gpu - dtheta| (t_k scale).
Full vectors at N <= 4096 (one to several FFT tiles plus the recurrence region);
sampled rows (oracle computes each row on its own) at N = 2^13 and 2^16, and at
the 4096 stored oracle rows at N = 2^20 and 2^22 (nodes here; the transforms
there in test_gpu_parity_large.py).
"""
import functools
import math

import numpy as np
import pytest

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


SMALL = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]


# --------------------------------------------------------------------------
# nodes and weights
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", SMALL)
def test_legpts_full(gb, N):
    x, th, w, dth = [host(t) for t in gb.Plan(N).legpts()]
    nd = onodes(N)
    ex = np.max(np.abs(x - nd.x))
    ew = np.max(np.abs(w - nd.w) / nd.w)
    et = np.max(np.abs(dth - nd["dtheta"])) * N
    eth = np.max(np.abs(th - nd.theta))
    print(f"N={N} x {ex:.2e} w {ew:.2e} t {et:.2e} theta {eth:.2e}")
    assert ex <= 4e-16
    assert ew <= 1e-14
    assert et <= 2e-14
    assert eth <= 1e-15
    # ordering: theta ascending, x descending
    assert np.all(np.diff(th) > 0) and np.all(np.diff(x) < 0)


@pytest.mark.parametrize("N", [2**13, 2**16, 2**20, 2**22])
def test_legpts_sampled(gb, N):
    """Nodes at sampled rows: 96 computed by the oracle at 2^13 and 2^16, the
    4096 stored oracle rows (tests/golden) at 2^20 and 2^22."""
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    p2 = int(math.log2(N))
    if N >= 2**20:
        import os
        z = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"rows4096_N2p{p2}.npz"))
        rows = z["rows"]
        nd = oracle.Nodes({k: z[k] for k in ("x_hi", "x_lo", "w_hi", "w_lo", "theta_hi", "theta_lo", "dtheta")})
    else:
        rows = inp.sample_rows(N, 96, seed=1000 + p2, include_ends=24)
        nd = onodes(N, tuple(rows.tolist()))
    x, th, w, dth = [host(t) for t in gb.Plan(N).legpts()]
    ex = np.max(np.abs(x[rows] - nd.x))
    ew = np.max(np.abs(w[rows] - nd.w) / nd.w)
    et = np.max(np.abs(dth[rows] - nd["dtheta"])) * N
    eth = np.max(np.abs(th[rows] - nd.theta))
    print(f"N={N} rows={rows.size} x {ex:.2e} w {ew:.2e} t {et:.2e} theta {eth:.2e}")
    assert ex <= 4e-16
    assert ew <= 1e-14
    assert et <= 2e-14
    assert eth <= 1e-15


# --------------------------------------------------------------------------
# transforms, full vectors
# --------------------------------------------------------------------------
def _c(N, seed, decay=0.0):
    import paper_1505_00354_gb300.inputs as inp
    return inp.coeffs(N, seed, decay)


@pytest.mark.parametrize("N", SMALL)
def test_leg2cheb_full(gb, N):
    import oracle
    c = _c(N, 1)
    got = host(gb.Plan(N, method=gb.METHOD_FAST).leg2cheb(dev(c)))
    err = np.max(np.abs(got - oracle.leg2cheb(c))) / np.abs(c).sum()
    print(f"N={N} leg2cheb err/||c||1 = {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("N", SMALL)
def test_chebeval_full(gb, N):
    import oracle
    c = _c(N, 2)
    got = host(gb.Plan(N, method=gb.METHOD_FAST).chebeval(dev(c)))
    ref = oracle.ndct_rows(c, onodes(N))
    err = np.max(np.abs(got - ref)) / np.abs(c).sum()
    print(f"N={N} chebeval err/||c||1 = {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("decay", [0.0, 1.0])
@pytest.mark.parametrize("N", SMALL)
def test_dlt_full(gb, N, decay):
    import oracle
    c = _c(N, 3, decay)
    got = host(gb.Plan(N, method=gb.METHOD_FAST).dlt(dev(c)))
    ref = oracle.dlt_rows(c, onodes(N))
    err = np.max(np.abs(got - ref)) / np.abs(c).sum()
    print(f"N={N} decay={decay} dlt err/||c||1 = {err:.2e}")
    assert err <= TOL64


def _idlt_err(got, ref, w, f):
    N = f.size
    scale = (np.arange(N) + 0.5) * np.abs(w * f).sum()
    return np.max(np.abs(got - ref) / scale)


@pytest.mark.parametrize("N", SMALL)
def test_idlt_full(gb, N):
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    f = inp.values(N, 4)
    nd = onodes(N)
    got = host(gb.Plan(N, method=gb.METHOD_FAST).idlt(dev(f)))
    ref = oracle.idlt(f, nd)
    err = _idlt_err(got, ref, nd.w, f)
    print(f"N={N} idlt err = {err:.2e} (abs {np.max(np.abs(got - ref)):.2e})")
    assert err <= TOL64


@pytest.mark.parametrize("N", [16, 256, 1024, 4096])
def test_idlt_dlt_roundtrip(gb, N):
    c = _c(N, 5)
    p = gb.Plan(N, method=gb.METHOD_FAST)
    back = host(p.idlt(p.dlt(dev(c))))
    err = np.max(np.abs(back - c)) / np.abs(c).sum()
    print(f"N={N} idlt(dlt(c)) - c: {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("N", [2, 8, 64, 512, 4096])
def test_transposes_full(gb, N):
    import oracle
    nd = onodes(N)
    g = _c(N, 6)
    p = gb.Plan(N, method=gb.METHOD_FAST)
    s = np.abs(g).sum()
    e1 = np.max(np.abs(host(p.dlt_t(dev(g))) - oracle.dlt_t(g, nd))) / s
    e2 = np.max(np.abs(host(p.chebeval_t(dev(g))) - oracle.ndct_t(g, nd))) / s
    e3 = np.max(np.abs(host(p.leg2cheb_t(dev(g))) - oracle.leg2cheb_t(g))) / s
    # idlt_t = D_w P D_s g
    ref4 = nd.w * oracle.dlt_rows((np.arange(N) + 0.5) * g, nd)
    e4 = np.max(np.abs(host(p.idlt_t(dev(g))) - ref4)) / np.abs((np.arange(N) + 0.5) * g).sum()
    print(f"N={N} dlt_t {e1:.2e} chebeval_t {e2:.2e} leg2cheb_t {e3:.2e} idlt_t {e4:.2e}")
    for e in (e1, e2, e3, e4):
        assert e <= TOL64


# --------------------------------------------------------------------------
# large N: sampled rows / residuals
# --------------------------------------------------------------------------
LARGE = [(2**13, 512), (2**16, 1024)]


@pytest.mark.parametrize("decay", [0.0, 1.0])
@pytest.mark.parametrize("N,nrows", LARGE)
def test_dlt_sampled(gb, N, nrows, decay):
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    p2 = int(math.log2(N))
    c = inp.coeffs(N, (10 if decay else 20) + p2, decay)
    rows = inp.sample_rows(N, nrows, seed=1000 + p2)
    got = host(gb.Plan(N, method=gb.METHOD_FAST).dlt(dev(c)))
    ref = oracle.dlt_rows(c, onodes(N, tuple(rows.tolist())))
    err = np.max(np.abs(got[rows] - ref)) / np.abs(c).sum()
    print(f"N={N} decay={decay} rows={rows.size} dlt err/||c||1 = {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("N,nrows", LARGE)
def test_idlt_forward_residual(gb, N, nrows):
    """IDLT above the full-oracle range: the exact inverse satisfies
    sum_n c_n P_n(x_k) = f_k, checked at sampled rows (residual / ||c||_1)."""
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    p2 = int(math.log2(N))
    f = inp.values(N, 30 + p2)
    rows = inp.sample_rows(N, nrows, seed=2000 + p2)
    c = host(gb.Plan(N, method=gb.METHOD_FAST).idlt(dev(f)))
    resid = oracle.dlt_rows(c, onodes(N, tuple(rows.tolist()))) - f[rows]
    err = np.max(np.abs(resid)) / np.abs(c).sum()
    print(f"N={N} idlt forward residual / ||c||1 = {err:.2e}")
    assert err <= TOL64


@pytest.mark.parametrize("N", [2**13, 2**16, 2**20])
def test_adjoint_identities(gb, N):
    """<A y, z> = <y, A^T z> for every operator pair, at sizes beyond the oracle."""
    import paper_1505_00354_gb300.inputs as inp
    p = gb.Plan(N, method=gb.METHOD_FAST)
    y, z = dev(inp.coeffs(N, 7)), dev(inp.coeffs(N, 8))
    for fwd, tr in ((p.dlt, p.dlt_t), (p.chebeval, p.chebeval_t), (p.leg2cheb, p.leg2cheb_t),
                    (p.idlt, p.idlt_t)):
        a = float(torch.dot(fwd(y), z))
        b = float(torch.dot(y, tr(z)))
        scale = float(torch.linalg.vector_norm(y, 1) * torch.linalg.vector_norm(z, 1))
        assert abs(a - b) <= 1e-13 * scale, (fwd.__name__, a, b)


@pytest.mark.parametrize("N", [2**12, 2**16, 2**20])
def test_input_scale_invariance(gb, N):
    """Scaling the input by 2^(+-700) scales every output by the same power of
    two: an FP64 plan's FP32 band vectors are normalised by the exponent of each
    item's largest input, so they neither overflow nor underflow."""
    import paper_1505_00354_gb300.inputs as inp
    p = gb.Plan(N, method=gb.METHOD_FAST)
    assert p.params()["M_fp32"] > 0
    x = dev(np.stack([inp.coeffs(N, 40), inp.coeffs(N, 41, 1.0)]))
    for op in (p.dlt, p.idlt, p.dlt_t, p.idlt_t, p.leg2cheb, p.leg2cheb_t):
        y = op(x)
        ref = float(torch.max(torch.abs(y)))
        for k in (-700, 700):
            ys = op(x * 2.0**k) * 2.0**-k
            err = float(torch.max(torch.abs(ys - y)))
            assert err <= 1e-14 * ref, (op.__name__, k, err, ref)


# --------------------------------------------------------------------------
# FP32 form
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [64, 1024, 4096])
def test_fp32_form_full(gb, N):
    import oracle
    c = _c(N, 9, 1.0)
    p = gb.Plan(N, gb.FP32, method=gb.METHOD_FAST)
    got = host(p.dlt(dev(c, torch.float32)))
    c32 = c.astype(np.float32).astype(np.float64)
    nd = onodes(N)
    err = np.max(np.abs(got - oracle.dlt_rows(c32, nd))) / np.abs(c32).sum()
    f = _c(N, 10)
    f32 = f.astype(np.float32).astype(np.float64)
    gi = host(p.idlt(dev(f, torch.float32)))
    ei = _idlt_err(gi, oracle.idlt(f32, nd), nd.w, f32)
    print(f"N={N} fp32 dlt {err:.2e} idlt {ei:.2e}")
    assert err <= TOL32 and ei <= TOL32


@pytest.mark.parametrize("p2", list(range(12, 23)))
@pytest.mark.parametrize("decay", [0.0, 1.0])
def test_fp32_form_sweep(gb, p2, decay):
    """The FP32 form across N = 2^12 .. 2^22, decaying and non-decaying c, against
    the FP64 oracle at sampled rows (all rows up to 2^14)."""
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    N = 2**p2
    c = inp.coeffs(N, 500 + p2 + int(10 * decay), decay).astype(np.float32).astype(np.float64)
    p = gb.Plan(N, gb.FP32, method=gb.METHOD_FAST)
    got = host(p.dlt(dev(c, torch.float32)))
    if N <= 2**14:
        rows = np.arange(N)
        nd = onodes(N)
    else:
        rows = inp.sample_rows(N, 32, seed=5000 + p2)
        nd = onodes(N, tuple(rows.tolist()))
    err = np.max(np.abs(got[rows] - oracle.dlt_rows(c, nd))) / np.abs(c).sum()
    print(f"N=2^{p2} decay {decay} fp32 dlt err/||c||1 = {err:.2e}")
    assert err <= TOL32


@pytest.mark.parametrize("eps", [1e-6, 1e-9, 1e-12])
@pytest.mark.parametrize("N", [4096, 2**16])
def test_general_eps(gb, eps, N):
    """A user tolerance (Sec. 3: parameters for an arbitrary eps): fewer Taylor
    terms for larger eps (the band layout and the precision of each expansion
    term follow the cost model and need not shrink monotonically), and the DLT
    within eps * ||c||_1."""
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    p = gb.Plan(N, eps=eps, method=gb.METHOD_FAST)
    q, q0 = p.params(), gb.plan_params(N, method=gb.METHOD_FAST)
    assert q["L"] <= q0["L"]
    c = inp.coeffs(N, 600 + N % 97, 0.0)
    got = host(p.dlt(dev(c)))
    rows = np.arange(N) if N <= 4096 else inp.sample_rows(N, 128, seed=601)
    nd = onodes(N) if N <= 4096 else onodes(N, tuple(rows.tolist()))
    err = np.max(np.abs(got[rows] - oracle.dlt_rows(c, nd))) / np.abs(c).sum()
    print(f"N={N} eps={eps:g}: L={q['L']} M={q['M']} K={q['K']} err/||c||1 = {err:.2e}")
    assert err <= eps


@pytest.mark.parametrize("N,nrows", [(2**16, 256)])
def test_fp32_form_sampled(gb, N, nrows):
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    p2 = int(math.log2(N))
    c = inp.coeffs(N, 40 + p2, 1.0).astype(np.float32).astype(np.float64)
    rows = inp.sample_rows(N, nrows, seed=3000 + p2)
    got = host(gb.Plan(N, gb.FP32, method=gb.METHOD_FAST).dlt(dev(c, torch.float32)))
    ref = oracle.dlt_rows(c, onodes(N, tuple(rows.tolist())))
    err = np.max(np.abs(got[rows] - ref)) / np.abs(c).sum()
    print(f"N={N} fp32 dlt err/||c||1 = {err:.2e}")
    assert err <= TOL32


# --------------------------------------------------------------------------
# batching, argument checks
# --------------------------------------------------------------------------
def test_batch_matches_single(gb):
    N = 1024
    p = gb.Plan(N, method=gb.METHOD_FAST)
    C = dev(np.stack([_c(N, 100 + i) for i in range(3)]))
    Fb = p.dlt(C)
    for i in range(3):
        assert torch.equal(Fb[i], p.dlt(C[i].clone()))
    empty = torch.empty(0, N, dtype=torch.float64, device="cuda")
    assert p.dlt(empty).shape == (0, N)


def test_argument_errors(gb):
    import ctypes
    L = gb.lib()
    h = ctypes.c_void_p()
    for bad in (0, 2**25):
        assert L.gbdlt_plan_create(bad, 0, 0.0, None, ctypes.byref(h)) == -2
    assert L.gbdlt_plan_create_ex(2**24 + 1, 0, 0.0, 1, None, ctypes.byref(h)) == -2
    assert L.gbdlt_plan_create_ex(2**17, 0, 0.0, 2, None, ctypes.byref(h)) == -2
    assert L.gbdlt_plan_create(64, 7, 0.0, None, ctypes.byref(h)) == -1
    # a direct-method plan for a length that is not a power of two has no
    # FFT-based chain: leg2cheb and chebeval are not open to it
    q = gb.Plan(1000, method=gb.METHOD_DIRECT)
    assert q.params()["method"] == 2 and q.params()["grid_n"] == 0
    y = torch.zeros(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbdltError):
        q.leg2cheb(y)
    # AUTO above 256 takes the chain on the next power-of-two grid
    assert gb.Plan(1000).params()["grid_n"] == 1024
    p = gb.Plan(64, method=gb.METHOD_FAST)
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert L.gbdlt_dlt(p.handle, None, ctypes.c_void_p(x.data_ptr()), 1) == -1
    assert L.gbdlt_dlt(p.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1) == -1
    assert L.gbdlt_dlt(p.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), -1) == -1
    assert L.gbdlt_plan_sync(p.handle) == 0


@pytest.mark.parametrize("op", ["dlt", "idlt", "dlt_t"])
def test_first_call_in_fresh_process(gb, op):
    """The first transform of a process may reach any FFT entry path first (the
    band FFTs take the four-step launcher directly): every path must set the
    kernels' shared-memory limits itself."""
    import subprocess
    import sys
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import torch, paper_1505_00354_gb300 as g; "
            "p = g.Plan(8192, method=g.METHOD_FAST); "
            f"y = p.{op}(torch.ones(8192, dtype=torch.float64, device='cuda')); "
            "torch.cuda.synchronize(); print(float(y.abs().sum()))")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]


def test_max_n(gb):
    """The largest N a plan accepts (2^24, FP64): sampled rows of the DLT against
    the oracle, and the IDLT's forward residual there."""
    import oracle
    import paper_1505_00354_gb300.inputs as inp
    N = 2**24
    p = gb.Plan(N, method=gb.METHOD_FAST)
    c = inp.coeffs(N, 924, 1.0)
    f = p.dlt(dev(c))
    # interior rows: the oracle's double-double Newton cannot settle the nodes
    # nearest x = +-1 at this N (its recurrence's rounding floor is above its stop
    # threshold there); those rows are checked at N <= 2^22
    rows = inp.sample_rows(N, 16, seed=925, include_ends=0)
    nd = onodes(N, tuple(rows.tolist()))
    err = np.max(np.abs(host(f)[rows] - oracle.dlt_rows(c, nd))) / np.abs(c).sum()
    cb = host(p.idlt(f))
    res = np.max(np.abs(oracle.dlt_rows(cb, nd) - host(f)[rows])) / np.abs(cb).sum()
    print(f"N=2^24: dlt {err:.2e}, idlt forward residual {res:.2e}")
    assert err <= TOL64 and res <= TOL64
    with pytest.raises(gb.GbdltError):
        gb.Plan(2 * N)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1024, 1 << 16, 1 << 20])
def test_side_branch_bitwise(gb, N, prec):
    """FP64 plans run their float-float and FP32 transforms on a side stream beside
    the FP64 work of the same stage; FP32 plans run their dense head blocks there.
    The results are bitwise those of the serial order (while the per-kernel
    profiler is on, every launch stays on one stream), for every operator, on the
    first (direct) call, the capturing call and graph replays, on the default
    stream and on a non-default one."""
    fp = gb.FP64 if prec == "fp64" else gb.FP32
    x = dev(_c(N, 91), torch.float64 if prec == "fp64" else torch.float32)
    ops = ["leg2cheb", "leg2cheb_t", "chebeval", "chebeval_t", "dlt", "dlt_t", "idlt", "idlt_t"]
    p = gb.Plan(N, fp, method=gb.METHOD_FAST)
    p.profile(1)
    ref = {op: getattr(p, op)(x).clone() for op in ops}
    p.profile(0)
    torch.cuda.synchronize()
    for op in ops:
        y = torch.empty_like(x)
        for _ in range(4):
            getattr(p, op)(x, out=y)
            torch.cuda.synchronize()
            assert torch.equal(y, ref[op]), op
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        q = gb.Plan(N, fp, method=gb.METHOD_FAST, stream=s)
        for op in ("dlt", "idlt"):
            y = torch.empty_like(x)
            for _ in range(3):
                getattr(q, op)(x, out=y)
            s.synchronize()
            assert torch.equal(y, ref[op]), op


def test_graph_replay(gb):
    """Repeated calls with the same pointers replay a captured chain: results are
    bitwise those of the direct run, on the default stream and on a side stream,
    and the launch count of a replay is the graph's kernel count."""
    N = 512
    for method in (gb.METHOD_FAST, gb.METHOD_DIRECT):
        p = gb.Plan(N, method=method)
        x = dev(_c(N, 77))
        y = torch.empty_like(x)
        outs = []
        for _ in range(5):
            p.dlt(x, out=y)
            outs.append(y.clone())
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        c0 = gb.launch_count()
        p.dlt(x, out=y)
        torch.cuda.synchronize()
        assert gb.launch_count() > c0
        assert torch.equal(y, outs[0])
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = gb.Plan(N, method=gb.METHOD_FAST, stream=s)
        x = dev(_c(N, 78))
        ref = p.idlt(x).clone()
        y = torch.empty_like(x)
        for _ in range(4):
            p.idlt(x, out=y)
        s.synchronize()
        assert torch.equal(y, ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [1 << 13, 1 << 16, 1 << 19, 1 << 20, 1 << 22])
def test_fft_staging_bitwise(gb, N, prec):
    """The FP32 FFT passes staged by the tensor memory accelerator compute the
    same butterflies in the same order as the per-thread-load passes: every
    operator's result is bitwise identical with staging on and off, for FP32
    plans and for the FP32 tier of FP64 plans (replays included)."""
    fp = gb.FP64 if prec == "fp64" else gb.FP32
    x = dev(_c(N, 93, 1.0), torch.float64 if prec == "fp64" else torch.float32)
    ops = ["leg2cheb", "leg2cheb_t", "chebeval", "chebeval_t", "dlt", "dlt_t", "idlt", "idlt_t"]
    p = gb.Plan(N, fp, method=gb.METHOD_FAST)
    p.set_fft_staging(False)
    ref = {op: getattr(p, op)(x).clone() for op in ops}
    p.set_fft_staging(True)
    # the default stays whatever the plan chose; both settings agree bitwise
    for op in ops:
        y = torch.empty_like(x)
        for _ in range(3):
            getattr(p, op)(x, out=y)
            assert torch.equal(y, ref[op]), op
    assert gb.lib().gbdlt_plan_sync(p.handle) == 0
    with pytest.raises(gb.GbdltError):
        gb._binding._check(gb.lib().gbdlt_plan_set_fft_staging(p.handle, 2), "set_fft_staging")


def test_fp64_rate_probe(gb):
    """The FP64 FMA-chain probe reaches a rate near the FP64 pipe's peak
    (2 FMA per SM and clock at up to 2070 MHz): the roofline denominator of the
    FP64 kernels is a measured number, not only a derived one."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 2 * 2 * 2.07e9
    r = gb.fp64_fma_rate()
    print(f"FP64 FMA probe: {r / 1e12:.4f} TFLOP/s ({r / peak:.3f} of {peak / 1e12:.4f} derived)")
    assert 0.3 * peak < r < 1.1 * peak


@pytest.mark.parametrize("N", [2**13, 2**16, 2**20])
def test_fft_mix_bitwise(gb, N):
    """The mixed FP64 / float-float Taylor FFT launches give bitwise the results
    of the two-stream launches (the same butterflies on the same data)."""
    import paper_1505_00354_gb300.inputs as inp
    p = gb.Plan(N, method=gb.METHOD_FAST)
    x = dev(np.stack([inp.coeffs(N, 60, 1.0), inp.coeffs(N, 61)]))
    ops = ("dlt", "idlt", "dlt_t", "idlt_t", "chebeval", "chebeval_t")
    p.set_fft_mix(0)
    ref = {op: getattr(p, op)(x).clone() for op in ops}
    p.set_fft_mix(2)
    for op in ops:
        assert torch.equal(getattr(p, op)(x), ref[op]), op
    p.set_fft_mix(1)  # the default: mixed from 2^20 up
    for op in ops:
        assert torch.equal(getattr(p, op)(x), ref[op]), op
    for bad in (-1, 3):
        with pytest.raises(gb.GbdltError):
            gb._binding._check(gb.lib().gbdlt_plan_set_fft_mix(p.handle, bad), "set_fft_mix")
