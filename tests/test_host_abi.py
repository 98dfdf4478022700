"""CPU-only checks of the C ABI library: it loads, exports every symbol the
header declares, and its host-side parameter derivation follows the paper's
bounds (Corollary 2.4 / Table 1 for L).  No compute call touches a GPU."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gb():
    from paper_1505_00354_gb300 import build
    build.build()
    import paper_1505_00354_gb300 as g
    return g


def header_functions():
    src = open(os.path.join(ROOT, "include", "gbdlt.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*|uint64_t)\s+(gbdlt_\w+)\s*\(", src, re.M)))


def test_exports_every_header_symbol(gb):
    names = header_functions()
    assert len(names) >= 17
    lib = gb.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(gb._binding.ENTRY_POINTS)


def test_status_strings(gb):
    lib = gb.lib()
    for code in range(-6, 1):
        s = lib.gbdlt_status_string(code)
        assert s and s != b"unknown status"
    assert lib.gbdlt_status_string(-99) == b"unknown status"


def test_launch_count_is_host_only(gb):
    assert gb.launch_count() >= 0


def test_bad_arguments(gb):
    lib = gb.lib()
    p = gb._binding.Params()
    for bad in (0, 2**25):
        assert lib.gbdlt_plan_params(bad, 0, 0.0, ctypes.byref(p)) == -2
    # the FFT-based chain takes any N in 1..2^24; the direct method N <= 65536
    for bad in (0, 2**24 + 1):
        assert lib.gbdlt_plan_params_ex(bad, 0, 0.0, 1, ctypes.byref(p)) == -2
    for bad in (65537, 2**17):
        assert lib.gbdlt_plan_params_ex(bad, 0, 0.0, 2, ctypes.byref(p)) == -2
    assert lib.gbdlt_plan_params_ex(64, 0, 0.0, 3, ctypes.byref(p)) == -1
    assert lib.gbdlt_plan_params(64, 2, 0.0, ctypes.byref(p)) == -1
    assert lib.gbdlt_plan_params(64, 0, 2.0, ctypes.byref(p)) == -1
    assert lib.gbdlt_plan_params(64, 0, 0.0, None) == -1
    assert lib.gbdlt_plan_destroy(None) == -1
    assert lib.gbdlt_plan_sync(None) == -1
    assert lib.gbdlt_dlt(None, None, None, 1) == -1


def test_method_selection(gb):
    """GBDLT_METHOD_AUTO: the direct method for N <= 256, the FFT-based chain
    otherwise (on the next power-of-two grid when N is not a power of two); the
    direct method's work is ceil(N/2) rows x N columns of the recurrence."""
    for N, m in ((1, 2), (3, 2), (256, 2), (257, 1), (1000, 1), (512, 1), (4096, 1), (2**20, 1), (10**6, 1)):
        q = gb.plan_params(N)
        assert q["method"] == m, N
        if m == 2:
            assert q["direct_steps"] == ((N + 1) // 2) * N
        if m == 2 and N & (N - 1):  # no FFT-based chain: no bands, no grid
            assert q["K"] == 0 and q["M"] == 0 and q["grid_n"] == 0
        if m == 1:
            assert q["grid_n"] == 1 << (N - 1).bit_length()
    assert gb.plan_params(1024, method=2)["method"] == 2
    assert gb.plan_params(1000, method=2)["grid_n"] == 0
    assert gb.plan_params(256, method=1)["method"] == 1
    assert gb.plan_params(2**17, method=1)["direct_steps"] == 0


@pytest.mark.parametrize("N", [3, 5, 100, 1000, 1025, 3000, 12345, 100000, 10**6, 2**20 - 1, 2**24 - 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_grid_plan_params(gb, N, prec):
    """N not a power of two: the chain of the grid G = 2^ceil(log2 N), whose band
    layout and head block are those of a plan for G; L from Corollary 2.4 with
    |n dtheta| <= (N-1) pi / (2G) (rows expanded about their nearest grid point)
    in place of 0.83845."""
    G = 1 << (N - 1).bit_length()
    q = gb.plan_params(N, prec, method=gb.METHOD_FAST)
    qG = gb.plan_params(G, prec, method=gb.METHOD_FAST)
    assert q["N"] == N and q["grid_n"] == G and q["method"] == gb.METHOD_FAST
    for key in ("K", "M", "bands", "head", "M_fp32", "M_ff"):
        assert q[key] == qG[key], key
    b = (N - 1) * math.pi / (2 * G) * (1 + 1e-9)
    eps = q["eps"]
    L = 1
    while b**L / math.factorial(L) > eps / 2 and L < 24:
        L += 1
    assert q["L"] == L
    # the worst row sits half a grid cell from its point: b is attained up to (N-1)/N
    assert q["L"] >= qG["L"] or b < 0.83845
    assert q["direct_steps"] == (((N + 1) // 2) * N if N <= 65536 else 0)


def _taylor_L(eps):
    # Corollary 2.4 (theta* = theta^cheb1): smallest L with 0.83845^L / L! <= eps/2
    L = 1
    while 0.83845**L / math.factorial(L) > eps / 2:
        L += 1
    return L


@pytest.mark.parametrize("eps,L_expected", [(1e-14, 16), (2e-6, 9), (4e-16, 17), (1e-7, 10)])
def test_taylor_terms_follow_table1(gb, eps, L_expected):
    """The Taylor term count is the smallest L whose Table 1 entry is below eps/2;
    Table 1 (Sec. 2.2) prints 1.4e-16 at L = 17 (double precision) and 4.7e-8
    at L = 10."""
    assert _taylor_L(eps) == L_expected
    assert gb.plan_params(1024, 0, eps)["L"] == L_expected


@pytest.mark.parametrize("N", [4, 64, 1024, 2**16, 2**20, 2**22])
@pytest.mark.parametrize("prec", [0, 1])
def test_band_layout_is_consistent(gb, N, prec):
    p = gb.plan_params(N, prec)
    bands = p["bands"]
    assert p["K"] == len(bands) <= 32
    H = N // 2
    prev_kb = None
    prev_ns = N + 1
    for ns, ka, kb in bands:
        assert 0 <= ka < kb <= H
        assert 2 <= ns <= N
        assert ns < prev_ns  # cuts shrink toward the middle rows
        if prev_kb is not None:
            assert ka == prev_kb  # contiguous
        prev_kb, prev_ns = kb, ns
    if bands:
        assert bands[-1][2] == H
        assert 1 <= p["M"] <= 24
    # dense head block: a multiple of the segment length, at most N/4, and no
    # band cuts below it
    h = p["head"]
    assert h == 0 or (h % p["seg_len"] == 0 and h <= N // 4)
    # segments of 512 columns (256 in FP32 plans); head sizes multiples of 512
    # in both precisions
    assert p["seg_len"] == (256 if p["prec"] == 1 else 512)
    assert h % 512 == 0
    assert all(ns >= h for ns, _, _ in bands)
    # recurrence work matches the layout (every row starts at n = head)
    k0 = bands[0][1] if bands else H
    steps = k0 * (N - h) + sum((kb - ka) * (ns - h) for ns, ka, kb in bands)
    assert p["rec_steps"] == 2 * steps
    # algorithmic bytes: c, dtheta in; f out (+ w for the IDLT)
    ds = 8 if prec == 0 else 4
    assert p["bytes_dlt"] == (2 * ds + 8) * N
    assert p["bytes_idlt"] == (2 * ds + 16) * N


def test_bands_respect_asymptotic_bound(gb):
    """Every band row satisfies the expansion's error bound at the band's cut:
    2 C_n h_{M,n} / (2 sin theta)^{M+1/2} <= eps/20 with n = ns at the band's
    first (worst) row."""
    for N in (1024, 2**16, 2**20):
        p = gb.plan_params(N, 0)
        M, eps = p["M"], p["eps"]
        for ns, ka, kb in p["bands"]:
            s = math.sin((ka + 0.5) * math.pi / N)
            lc = 0.5 * math.log(4 / math.pi) + math.lgamma(ns + 1) - math.lgamma(ns + 1.5)
            lh = sum(2 * math.log(j - 0.5) - math.log(j) - math.log(ns + j + 0.5) for j in range(1, M + 1))
            bound = 2 * math.exp(lc + lh) / (2 * s) ** (M + 0.5)
            assert bound <= eps / 20 * (1 + 1e-9), (N, ns, ka, bound)


@pytest.mark.parametrize("N", [1024, 2**16, 2**20, 2**22])
def test_precision_tiers_within_budget(gb, N):
    """FP64 plans run the tail of each band's expansion in FP32 and the terms
    before it in float-float: on every band the FFT rounding of those terms,
    2 log2(N) u T_m with T_m = 2 C_ns h_{m,ns} / (2 sin theta_ka)^{m+1/2} (the
    term's bound at the band's first row; u = 2^-24 for FP32, 2^-46 for
    float-float), sums to at most eps/20 per tier; likewise the float-float
    Taylor terms l >= L - L_ff with T_l = 0.83845^l / l! (Corollary 2.4)."""
    p = gb.plan_params(N, 0)
    M, eps = p["M"], p["eps"]
    Mh = M - p["M_fp32"]
    M64 = Mh - p["M_ff"]
    assert 1 <= M64 <= Mh <= M
    lg = int(round(math.log2(N)))
    for ns, ka, kb in p["bands"]:
        s2 = 2 * math.sin((ka + 0.5) * math.pi / N)
        lc = 0.5 * math.log(4 / math.pi) + math.lgamma(ns + 1) - math.lgamma(ns + 1.5)

        def T(m):
            lh = sum(2 * math.log(j - 0.5) - math.log(j) - math.log(ns + j + 0.5) for j in range(1, m + 1))
            return 2 * math.exp(lc + lh) / s2 ** (m + 0.5)

        e32 = sum(2 * lg * 2.0**-24 * T(m) for m in range(Mh, M))
        eff = sum(2 * lg * 2.0**-46 * T(m) for m in range(M64, Mh))
        assert e32 <= eps / 20 * (1 + 1e-9), (N, ns, e32)
        assert eff <= eps / 20 * (1 + 1e-9), (N, ns, eff)
    L = p["L"]
    Lff = L - p["L_ff"]
    eL = sum(2 * lg * 2.0**-46 * 0.83845**l / math.factorial(l) for l in range(Lff, L))
    assert eL <= eps / 20 * (1 + 1e-9)
    # FP32 plans have no tiers
    q = gb.plan_params(N, 1)
    assert q["M_fp32"] == 0 and q["M_ff"] == 0 and q["L_ff"] == 0
