"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against mathematics the paper states or relies on:
closed-form nodes and weights, Gauss exactness, the node-distance bounds of
Lemma 2.3, the change of basis P = T M of Sec. 3, the discrete orthogonality of
Sec. 4, exact error-free transformations, and an independent multiprecision
library where one is available.  A dropped term, a wrong sign or index, or a
transposed operand in any oracle function fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

rng = np.random.default_rng(12345)


# --------------------------------------------------------------------------
# double-double arithmetic
# --------------------------------------------------------------------------
def test_two_prod_two_sum_exact(orc):
    for _ in range(200):
        a, b = rng.standard_normal(2) * 10.0 ** rng.integers(-20, 20, 2)
        hi, lo = orc.two_prod(a, b)
        assert Fraction(hi) + Fraction(lo) == Fraction(a) * Fraction(b)
        hi, lo = orc.two_sum(a, b)
        assert Fraction(hi) + Fraction(lo) == Fraction(a) + Fraction(b)


def test_dd_div_sqrt(orc):
    for _ in range(100):
        a = (float(rng.standard_normal()), float(rng.standard_normal()) * 1e-17)
        b = (float(rng.uniform(0.5, 3.0)), float(rng.standard_normal()) * 1e-17)
        q = orc.dd_div(a, b)
        A = Fraction(a[0]) + Fraction(a[1])
        B = Fraction(b[0]) + Fraction(b[1])
        Q = Fraction(q[0]) + Fraction(q[1])
        assert abs(float((Q - A / B) / (A / B))) < 1e-30
        s = orc.dd_sqrt((abs(a[0]), 0.0))
        S = Fraction(s[0]) + Fraction(s[1])
        assert abs(float((S * S - Fraction(abs(a[0]))) / Fraction(abs(a[0])))) < 1e-30


def test_sincos_dd(orc):
    # sin^2 + cos^2 = 1 to dd accuracy, and agreement with a multiprecision library
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for _ in range(50):
        t = float(rng.uniform(0.0, math.pi))
        (sh, sl), (ch, cl) = orc.sincos_dd(t, 0.0)
        S = Fraction(sh) + Fraction(sl)
        C = Fraction(ch) + Fraction(cl)
        assert abs(float(S * S + C * C - 1)) < 1e-30
        assert abs(float(mp.mpf(sh) + mp.mpf(sl) - mp.sin(mp.mpf(t)))) < 1e-30
        assert abs(float(mp.mpf(ch) + mp.mpf(cl) - mp.cos(mp.mpf(t)))) < 1e-30


# --------------------------------------------------------------------------
# polynomials
# --------------------------------------------------------------------------
def test_legendre_endpoints(orc):
    for n in [0, 1, 2, 7, 64, 1000, 4097]:
        assert orc.legendre_p(n, [1.0])[0] == pytest.approx(1.0, abs=1e-14)
        assert orc.legendre_p(n, [-1.0])[0] == pytest.approx((-1.0) ** n, abs=1e-14)


def test_legendre_closed_forms(orc):
    x = rng.uniform(-1, 1, 64)
    closed = {
        0: np.ones_like(x),
        1: x,
        2: (3 * x**2 - 1) / 2,
        3: (5 * x**3 - 3 * x) / 2,
        4: (35 * x**4 - 30 * x**2 + 3) / 8,
        5: (63 * x**5 - 70 * x**3 + 15 * x) / 8,
    }
    for n, ref in closed.items():
        np.testing.assert_allclose(orc.legendre_p(n, x), ref, rtol=0, atol=2e-15)


def test_legendre_vs_mpmath(orc):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x = rng.uniform(-1, 1, 8)
    for n in [50, 777, 3000]:
        got = orc.legendre_p(n, x)
        ref = np.array([float(mp.legendre(n, mp.mpf(v))) for v in x])
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-15)


def test_chebyshev_is_cos(orc):
    t = rng.uniform(0, math.pi, 64)
    for n in [0, 1, 2, 5, 33]:
        np.testing.assert_allclose(orc.chebyshev_t(n, np.cos(t)), np.cos(n * t), atol=1e-13)


# --------------------------------------------------------------------------
# nodes and weights
# --------------------------------------------------------------------------
CLOSED_NODES = {
    1: ([0.0], [2.0]),
    2: ([1 / math.sqrt(3), -1 / math.sqrt(3)], [1.0, 1.0]),
    3: ([math.sqrt(3 / 5), 0.0, -math.sqrt(3 / 5)], [5 / 9, 8 / 9, 5 / 9]),
    4: (
        [math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5)), math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)),
         -math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)), -math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))],
        [(18 - math.sqrt(30)) / 36, (18 + math.sqrt(30)) / 36,
         (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36],
    ),
    5: (
        [math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3, math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, 0.0,
         -math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, -math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3],
        [(322 - 13 * math.sqrt(70)) / 900, (322 + 13 * math.sqrt(70)) / 900, 128 / 225,
         (322 + 13 * math.sqrt(70)) / 900, (322 - 13 * math.sqrt(70)) / 900],
    ),
}


@pytest.mark.parametrize("N", sorted(CLOSED_NODES))
def test_legpts_closed_forms(orc, N):
    nd = orc.legpts(N)
    x_ref, w_ref = CLOSED_NODES[N]
    np.testing.assert_allclose(nd.x, x_ref, atol=1e-15)
    np.testing.assert_allclose(nd.w, w_ref, atol=1e-15)


@pytest.mark.parametrize("N", [37, 100])
def test_legpts_vs_scipy(orc, N):
    sp = pytest.importorskip("scipy.special")
    xs, ws = sp.roots_legendre(N)
    nd = orc.legpts(N)
    np.testing.assert_allclose(nd.x, xs[::-1], atol=4e-16)
    # scipy's weights carry about 1e-12 relative error (its nodes are better)
    np.testing.assert_allclose(nd.w, ws[::-1], rtol=1e-11)


@pytest.mark.parametrize("degree", [2, 4, 6])
def test_legpts_vs_mpmath_gauss_legendre(orc, degree):
    """mpmath's own Gauss-Legendre rule (3 * 2^(degree-1) points, 40 digits)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rule = mp.calculus.quadrature.GaussLegendre(mp.mp).calc_nodes(degree, mp.mp.prec)
    rule = sorted(rule, key=lambda t: -t[0])
    N = len(rule)
    nd = orc.legpts(N)
    for k, (xr, wr) in enumerate(rule):
        x = mp.mpf(nd["x_hi"][k]) + mp.mpf(nd["x_lo"][k])
        w = mp.mpf(nd["w_hi"][k]) + mp.mpf(nd["w_lo"][k])
        assert abs(x - xr) < mp.mpf("1e-26"), (N, k)
        assert abs(w - wr) < mp.mpf("1e-26") * wr, (N, k)


@pytest.mark.parametrize("N", [6, 64, 255, 1024])
def test_gauss_exactness(orc, N):
    nd = orc.legpts(N)
    assert abs(nd.w.sum() - 2.0) < 1e-14
    np.testing.assert_allclose(nd.x, -nd.x[::-1], atol=1e-16)
    np.testing.assert_allclose(nd.w, nd.w[::-1], rtol=1e-14)
    for j in sorted({0, 1, 2, 3, N - 1, N, 2 * N - 2, 2 * N - 1}):
        got = float(np.dot(nd.w, orc.legendre_p(j, nd.x)))
        assert got == pytest.approx(2.0 if j == 0 else 0.0, abs=5e-15), (N, j)
    # degree 2N is no longer integrated exactly: the weights are not a trivially
    # "right" answer for every degree
    got = float(np.dot(nd.w, orc.legendre_p(2 * N, nd.x)))
    assert abs(got) > 1e-6


@pytest.mark.parametrize("N", [8, 33, 1000, 4096])
def test_lemma_2_3_bounds(orc, N):
    """Lemma 2.3: 0 < theta^leg_k - theta^cheb*_k <= 1/(3pi(2N+1)) for k < N/2 and
    |theta^leg_k - theta^cheb1_k| <= (3pi^2+2)/(6pi(2N+1)) <= 0.83845/N."""
    nd = orc.legpts(N)
    k = np.arange(N)
    th_star = (k + 0.75) * np.pi / (N + 0.5)
    d_star = nd.theta - th_star
    half = N // 2
    assert np.all(d_star[:half] > 0)
    assert np.all(np.abs(d_star) <= 1 / (3 * np.pi * (2 * N + 1)) * (1 + 1e-12))
    bound1 = (3 * np.pi**2 + 2) / (6 * np.pi * (2 * N + 1))
    assert np.all(np.abs(nd["dtheta"]) <= bound1 * (1 + 1e-12))
    assert bound1 <= 0.83845 / N
    # dtheta is theta - (k+1/2)pi/N
    np.testing.assert_allclose(nd["dtheta"], nd.theta - (k + 0.5) * np.pi / N, atol=1e-15)


def test_lemma_2_3_tight(orc):
    """Fig. 2 reports the bounds of Lemma 2.3 as tight."""
    N = 4096
    nd = orc.legpts(N)
    k = np.arange(N)
    r1 = np.max(np.abs(nd["dtheta"])) / ((3 * np.pi**2 + 2) / (6 * np.pi * (2 * N + 1)))
    rs = np.max(np.abs(nd.theta - (k + 0.75) * np.pi / (N + 0.5))) * 3 * np.pi * (2 * N + 1)
    assert 0.98 < r1 <= 1.0
    assert 0.85 < rs <= 1.0


def test_legpts_sampled_large(orc):
    """Sampled nodes at N = 2^20 obey Lemma 2.3 and are roots of P_N."""
    N = 2**20
    ks = np.array([0, 1, 2, 17, 4097, N // 2 - 1, N // 2, N - 1], dtype=np.int64)
    nd = orc.legpts(N, ks)
    assert np.all(np.abs(nd["dtheta"]) * N <= 0.83845)
    # symmetry: theta_{N-1-k} = pi - theta_k
    a = orc.legpts(N, np.array([3], dtype=np.int64))
    b = orc.legpts(N, np.array([N - 4], dtype=np.int64))
    assert abs((a.theta[0] + b.theta[0]) - math.pi) < 1e-15
    assert abs(a.w[0] - b.w[0]) < 1e-15 * a.w[0]


# --------------------------------------------------------------------------
# DLT / IDLT / NDCT definitions
# --------------------------------------------------------------------------
def test_dlt_unit_vectors(orc):
    N = 64
    nd = orc.legpts(N)
    for n in [0, 1, 5, N - 1]:
        e = np.zeros(N)
        e[n] = 1.0
        np.testing.assert_allclose(orc.dlt_rows(e, nd), orc.legendre_p(n, nd.x), atol=2e-15)
    np.testing.assert_allclose(orc.dlt_rows(np.eye(N)[0], nd), np.ones(N), atol=0)


def test_dlt_closed_form_n3(orc):
    nd = orc.legpts(3)
    c = rng.standard_normal(3)
    x = np.array(CLOSED_NODES[3][0])
    ref = c[0] + c[1] * x + c[2] * (3 * x**2 - 1) / 2
    np.testing.assert_allclose(orc.dlt_rows(c, nd), ref, atol=1e-15)


def test_dlt_linear(orc):
    N = 100
    nd = orc.legpts(N)
    a, b = rng.standard_normal(N), rng.standard_normal(N)
    np.testing.assert_allclose(orc.dlt_rows(2 * a - 3 * b, nd),
                               2 * orc.dlt_rows(a, nd) - 3 * orc.dlt_rows(b, nd), atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 7, 256, 1024])
def test_idlt_inverts_dlt(orc, N):
    nd = orc.legpts(N)
    c = rng.standard_normal(N)
    f = orc.dlt_rows(c, nd)
    np.testing.assert_allclose(orc.idlt(f, nd), c, atol=2e-14)


def test_idlt_rows_partition(orc):
    """The row contributions of a partition of the nodes add up to the IDLT."""
    N = 96
    nd = orc.legpts(N)
    f = rng.standard_normal(N)
    parts = [np.arange(0, 30), np.arange(30, 31), np.arange(31, N)]
    tot = np.zeros(N)
    for r in parts:
        sub = {k: nd[k][r] for k in ("x_hi", "x_lo", "w_hi", "w_lo")}
        tot += orc.idlt_rows(f[r], sub, N)
    np.testing.assert_allclose(tot, orc.idlt(f, nd), atol=1e-14)


def test_idlt_simple_functions(orc):
    N = 50
    nd = orc.legpts(N)
    e0 = np.zeros(N)
    e0[0] = 1
    e1 = np.zeros(N)
    e1[1] = 1
    np.testing.assert_allclose(orc.idlt(np.ones(N), nd), e0, atol=1e-15)
    np.testing.assert_allclose(orc.idlt(nd.x, nd), e1, atol=1e-15)


def test_discrete_orthogonality(orc):
    """Sec. 4: P^T D_w P = D_s^{-1}, s_n = n + 1/2."""
    N = 40
    nd = orc.legpts(N)
    for j in [0, 3, N - 1]:
        e = np.zeros(N)
        e[j] = 1
        col = orc.dlt_t(nd.w * orc.dlt_rows(e, nd), nd)
        ref = np.zeros(N)
        ref[j] = 1 / (j + 0.5)
        np.testing.assert_allclose(col, ref, atol=1e-15)


def test_ndct_unit_vectors(orc):
    N = 128
    nd = orc.legpts(N)
    for n in [0, 1, 2, 77, N - 1]:
        e = np.zeros(N)
        e[n] = 1
        np.testing.assert_allclose(orc.ndct_rows(e, nd), np.cos(n * nd.theta), atol=1e-13)


# --------------------------------------------------------------------------
# Legendre -> Chebyshev matrix M (Sec. 3)
# --------------------------------------------------------------------------
def test_m_small_entries(orc):
    M = orc.leg2cheb_matrix(6)
    # P_2 = 1/4 T_0 + 3/4 T_2, P_3 = 3/8 T_1 + 5/8 T_3, P_1 = T_1, P_0 = T_0
    np.testing.assert_allclose(M[:, 0], [1, 0, 0, 0, 0, 0], atol=1e-16)
    np.testing.assert_allclose(M[:, 1], [0, 1, 0, 0, 0, 0], atol=1e-16)
    np.testing.assert_allclose(M[:, 2], [0.25, 0, 0.75, 0, 0, 0], atol=1e-16)
    np.testing.assert_allclose(M[:, 3], [0, 0.375, 0, 0.625, 0, 0], atol=1e-16)
    assert np.all(np.tril(M, -1) == 0)


def test_m_is_change_of_basis(orc):
    """P_n(x) = sum_k M_{kn} T_k(x) with T_k(x) = cos(k arccos x)."""
    N = 300
    M = orc.leg2cheb_matrix(N)
    x = rng.uniform(-1, 1, 20)
    T = np.cos(np.outer(np.arccos(x), np.arange(N)))
    for n in [0, 1, 2, 9, 150, N - 1]:
        np.testing.assert_allclose(T @ M[:, n], orc.legendre_p(n, x), atol=1e-13)


def test_leg2cheb_matches_matrix_and_transpose(orc):
    N = 200
    M = orc.leg2cheb_matrix(N)
    c, y = rng.standard_normal(N), rng.standard_normal(N)
    np.testing.assert_allclose(orc.leg2cheb(c), M @ c, atol=1e-13)
    np.testing.assert_allclose(orc.leg2cheb_t(y), M.T @ y, atol=1e-13)


def test_eq14_change_of_basis_on_nodes(orc):
    """Eq. 14: sum_n c_n P_n(x_k) = sum_n chat_n T_n(x_k), chat = M c."""
    N = 512
    nd = orc.legpts(N)
    c = rng.standard_normal(N)
    np.testing.assert_allclose(orc.ndct_rows(orc.leg2cheb(c), nd), orc.dlt_rows(c, nd), atol=1e-12)


# --------------------------------------------------------------------------
# transposes (adjoint identity)
# --------------------------------------------------------------------------
def test_adjoints(orc):
    N = 96
    nd = orc.legpts(N)
    y, z = rng.standard_normal(N), rng.standard_normal(N)
    assert np.dot(orc.leg2cheb(y), z) == pytest.approx(np.dot(y, orc.leg2cheb_t(z)), abs=1e-12)
    assert np.dot(orc.ndct_rows(y, nd), z) == pytest.approx(np.dot(y, orc.ndct_t(z, nd)), abs=1e-12)
    assert np.dot(orc.dlt_rows(y, nd), z) == pytest.approx(np.dot(y, orc.dlt_t(z, nd)), abs=1e-12)
    # IDLT = D_s P^T D_w
    s = np.arange(N) + 0.5
    np.testing.assert_allclose(orc.idlt(z, nd), s * orc.dlt_t(nd.w * z, nd), atol=1e-13)


# --------------------------------------------------------------------------
# Table 1 (the paper's printed numbers)
# --------------------------------------------------------------------------
def test_table1_values():
    """The printed values of Table 1 equal 0.83845^L/L! and ((6pi)^L L!)^-1 to the
    two digits shown, and the (3pi^2+2)/(12pi) constant of Lemma 2.3 rounds to
    0.83845."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_taylor_bounds.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 18
    for L, a, b in rows:
        L = int(L)
        va = 0.83845**L / math.factorial(L)
        vb = 1.0 / ((6 * math.pi) ** L * math.factorial(L))
        for printed, val in ((float(a), va), (float(b), vb)):
            ulp = 10.0 ** (math.floor(math.log10(printed)) - 1)
            assert abs(val - printed) <= 1.01 * ulp, (L, printed, val)
    assert round((3 * math.pi**2 + 2) / (12 * math.pi), 5) == 0.83845


# --------------------------------------------------------------------------
# plain FP64 direct method (the timed CPU baseline)
# --------------------------------------------------------------------------
U64 = 2.0**-53


@pytest.mark.parametrize("N", [2, 3, 5])
def test_f64_legpts_closed_forms(orc, N):
    """Nodes and weights of the FP64 Newton solve against the closed forms."""
    closed = {2: ([1 / math.sqrt(3), -1 / math.sqrt(3)], [1.0, 1.0]),
              3: ([math.sqrt(0.6), 0.0, -math.sqrt(0.6)], [5 / 9, 8 / 9, 5 / 9]),
              5: ([math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3, math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, 0.0,
                   -math.sqrt(5 - 2 * math.sqrt(10 / 7)) / 3, -math.sqrt(5 + 2 * math.sqrt(10 / 7)) / 3],
                  [(322 - 13 * math.sqrt(70)) / 900, (322 + 13 * math.sqrt(70)) / 900, 128 / 225,
                   (322 + 13 * math.sqrt(70)) / 900, (322 - 13 * math.sqrt(70)) / 900])}
    nd = orc.legpts_f64(N)
    x, w = closed[N]
    assert np.max(np.abs(nd["x"] - x)) <= 4 * U64
    assert np.max(np.abs(nd["w"] - w)) <= 16 * U64


@pytest.mark.parametrize("N", [7, 64, 255, 1000])
def test_f64_legpts_vs_scipy_and_dd(orc, N):
    """The FP64 solve against scipy's nodes and the dd oracle: x to a few u,
    theta to N u, w to N^2 u relative (x_k rounded to double moves P'_N by up to
    N^2 u near the ends, which is the plain FP64 method's error, not a defect).
    scipy's weights are not used: they differ from the mpmath-pinned dd weights
    by ~1e-8 at N = 1000."""
    sp = pytest.importorskip("scipy.special")
    nd = orc.legpts_f64(N)
    xs, _ = sp.roots_legendre(N)
    assert np.max(np.abs(nd["x"] - xs[::-1])) <= 1e-14
    dd = orc.legpts(N)
    assert np.max(np.abs(nd["x"] - dd.x)) <= 4 * U64
    assert np.max(np.abs(nd["theta"] - dd.theta)) <= (N + 16) * U64
    assert np.max(np.abs(nd["w"] - dd.w) / dd.w) <= (N * N + 64) * U64
    assert np.all(np.diff(nd["theta"]) > 0)


def test_f64_dlt_unit_vectors(orc):
    """c = e_n gives P_n at the nodes (scipy's Legendre values); c = e_0 gives 1."""
    sp = pytest.importorskip("scipy.special")
    N = 200
    x = orc.legpts_f64(N)["x"]
    for n in (0, 1, 2, 17, 100, N - 1):
        c = np.zeros(N)
        c[n] = 1.0
        f = orc.dlt_rows_f64(c, x)
        assert np.max(np.abs(f - sp.eval_legendre(n, x))) <= (n * n + 16) * U64
    c = np.zeros(N)
    c[0] = 1.0
    assert np.all(orc.dlt_rows_f64(c, x) == 1.0)


@pytest.mark.parametrize("N", [16, 512, 4096])
def test_f64_direct_vs_dd(orc, N):
    """Eq. 1 and Eq. 2 in plain FP64 against the dd oracle on the same (dd)
    nodes, within the FP64 method's bound N^2 u (the sensitivity of P_n to the
    rounding of x_k, |P'_n| <= n(n+1)/2, dominates the recurrence's own rounding)."""
    r = np.random.default_rng(N)
    c = r.standard_normal(N)
    nd = orc.legpts(N)
    f_dd = orc.dlt_rows(c, nd)
    f_64 = orc.dlt_rows_f64(c, nd.x)
    assert np.max(np.abs(f_64 - f_dd)) <= N * N * U64 * np.abs(c).sum()
    c_dd = orc.idlt(f_dd, nd)
    c_64 = orc.idlt_rows_f64(f_dd, nd.x, nd.w, N)
    scale = (np.arange(N) + 0.5) * np.abs(nd.w * f_dd).sum()
    assert np.max(np.abs(c_64 - c_dd) / scale) <= N * N * U64


@pytest.mark.parametrize("N", [8, 333, 2048])
def test_f64_direct_roundtrip(orc, N):
    """IDLT(DLT(c)) = c with the FP64 method's own nodes and weights, and the
    row partition: contributions of disjoint row sets add up to the whole."""
    r = np.random.default_rng(7 * N)
    c = r.standard_normal(N)
    nd = orc.legpts_f64(N)
    f = orc.dlt_rows_f64(c, nd["x"])
    back = orc.idlt_rows_f64(f, nd["x"], nd["w"], N)
    assert np.max(np.abs(back - c)) <= N * N * U64 * np.abs(c).sum()
    half = N // 2
    a = orc.idlt_rows_f64(f[:half], nd["x"][:half], nd["w"][:half], N)
    b = orc.idlt_rows_f64(f[half:], nd["x"][half:], nd["w"][half:], N)
    assert np.max(np.abs(a + b - back)) <= 64 * U64 * np.abs(back).max() + 1e-300


# --------------------------------------------------------------------------
# restrictions to listed indices (the sampled-row and sparse-input checks)
# --------------------------------------------------------------------------
def test_rows_restrictions_match_full(orc):
    """Every *_rows function equals its full counterpart at the listed indices
    (leg2cheb), or on an input that is zero off the listed nodes (transposes),
    and contributions of a partition of the nodes add up to the full sum."""
    N = 300
    r = np.random.default_rng(3)
    nd = orc.legpts(N)
    ks = np.sort(r.choice(N, 37, replace=False))
    sub = orc.legpts(N, ks)
    g = r.standard_normal(ks.size)
    dense = np.zeros(N)
    dense[ks] = g
    for part, full in ((orc.dlt_t_rows(g, sub, N), orc.dlt_t(dense, nd)),
                       (orc.ndct_t_rows(g, sub, N), orc.ndct_t(dense, nd))):
        assert np.max(np.abs(part - full)) <= 1e-14 * np.abs(full).max()
    rest = np.setdiff1d(np.arange(N), ks)
    gr = r.standard_normal(rest.size)
    both = np.zeros(N)
    both[ks], both[rest] = g, gr
    s = orc.dlt_t_rows(g, sub, N) + orc.dlt_t_rows(gr, orc.legpts(N, rest), N)
    assert np.max(np.abs(s - orc.dlt_t(both, nd))) <= 1e-14 * np.abs(s).max()
    c = r.standard_normal(N)
    assert np.max(np.abs(orc.leg2cheb_rows(c, ks) - orc.leg2cheb(c)[ks])) <= 1e-15 * np.abs(c).sum()
    assert np.max(np.abs(orc.leg2cheb_t_rows(c, ks) - orc.leg2cheb_t(c)[ks])) <= 1e-15 * np.abs(c).sum()


def test_recurrence_coefficient_form(orc):
    """The dd recurrence with tabulated (2m+1)/(m+1), m/(m+1) keeps P_n exact
    at the closed forms and the end points for large n (P_n(1) = 1,
    P_n(-1) = (-1)^n, P_{2m}(0) = (-1)^m (2m)!/(4^m m!^2))."""
    for n in (1, 2, 3, 1000, 4097):
        assert orc.legendre_p(n, [1.0])[0] == 1.0
        assert orc.legendre_p(n, [-1.0])[0] == (-1.0) ** n
    for m in (1, 5, 50, 500):
        exact = Fraction((-1) ** m * math.comb(2 * m, m), 4**m)
        assert abs(orc.legendre_p(2 * m, [0.0])[0] - float(exact)) <= 2e-16 * abs(float(exact))


def test_legendre_p_at_dd_points(orc):
    """P_n at dd points: equals the double-point routine when x_lo = 0, and at
    the dd Gauss-Legendre nodes P_N vanishes to dd rounding (they are its
    roots) while P_{N-1} does not."""
    x = np.linspace(-1, 1, 41)
    for n in (0, 1, 7, 300):
        got = orc.legendre_p_at(n, {"x_hi": x, "x_lo": np.zeros_like(x)})
        assert np.array_equal(got, orc.legendre_p(n, x))
    N = 257
    nd = orc.legpts(N)
    assert np.max(np.abs(orc.legendre_p_at(N, nd))) <= 1e-25
    assert np.min(np.abs(orc.legendre_p_at(N - 1, nd))) >= 1e-3
