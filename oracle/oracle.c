/*
 * Oracle for the discrete Legendre transform (Hale & Townsend, "A fast
 * FFT-based discrete Legendre transform").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU definition of every quantity the GPU library computes.  Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library and must never sit on the product path.
 *
 * Arithmetic: double-double ("dd", about 106 significand bits) built from the
 * error-free transformations TwoSum (Knuth) and TwoProd through fma (Dekker's
 * product written with a fused multiply-add).  Inputs and outputs are IEEE
 * doubles; a dd value is returned as a (hi, lo) pair where the caller needs the
 * extra bits (nodes, weights).  The paper's "extended precision" reference
 * (Sec. 2.5, Sec. 3.1, Sec. 4.1) is read as double-double.
 *
 * What each function follows:
 *   orc_legendre_p   three-term recurrence (n+1)P_{n+1} = (2n+1)xP_n - nP_{n-1}
 *                    (textbook; the recurrence the paper's direct approach
 *                    uses, Sec. 2.4 and Sec. 4.1)
 *   orc_legpts       roots of P_N (Eq. 1): Newton in theta = arccos x, started
 *                    at the cheb* point (k+3/4)pi/(N+1/2) (Sec. 2.2), with P_N
 *                    and P_{N-1} from the recurrence; Gauss-Legendre weights
 *                    w = 2/(dP_N/dtheta)^2 at the root (textbook identity, the
 *                    paper only names the weights, Eq. 2)
 *   orc_dlt_rows     f_k = sum_n c_n P_n(x_k), Eq. 1, by the recurrence
 *   orc_dlt_t        (P^T g)_n = sum_k g_k P_n(x_k), Sec. 4 matrix form
 *   orc_idlt         c_n = (n+1/2) sum_k w_k f_k P_n(x_k), Eq. 2 ("along rows",
 *                    Sec. 4.1)
 *   orc_ndct_rows    f_k = sum_n c_n T_n(x_k), Eq. 3, by the Chebyshev
 *                    recurrence of Sec. 2.4
 *   orc_ndct_t       (T^T g)_n = sum_k g_k T_n(x_k), Sec. 4 item 2
 *   orc_leg2cheb     chat = M c with the Alpert-Rokhlin matrix of Sec. 3,
 *                    read with the Lambda-product entries (the printed
 *                    entries drop two Gamma factors; see the reading below)
 *   orc_leg2cheb_t   M^T y
 *   *_rows variants  the same sums restricted to listed output indices
 *                    (orc_leg2cheb_rows, orc_leg2cheb_t_rows) or to listed
 *                    nodes (orc_dlt_t_rows, orc_ndct_t_rows: the transposes
 *                    of an input that vanishes off those nodes)
 *   orc_cos_dd       cos/sin of a dd angle (argument reduction by dd pi/2 and
 *                    Taylor series), used for x_k = cos(theta_k)
 *   orc_legpts_f64,  the plain FP64 direct method (no double-double anywhere):
 *   orc_dlt_rows_f64, nodes by Newton on P_N from the cheb* point, Eq. 1 rows
 *   orc_idlt_rows_f64 and the rows' contributions to Eq. 2, every sum by the
 *                    three-term recurrence in double.  This is the baseline the
 *                    GPU path is timed against (the paper's direct approach,
 *                    Sec. 2.4 and Sec. 4.1); its error grows like N^2 u near
 *                    x = +-1 (the rounding of x_k alone moves P_n by up to
 *                    n^2 u / 2 there), so the dd functions above stay the
 *                    reference for accuracy.
 *
 * Reading of the matrix M (Sec. 3): with Lambda(z) = Gamma(z+1/2)/Gamma(z+1),
 *   M_{0n} = (1/pi) Lambda(n/2)^2                       n even,
 *   M_{kn} = (2/pi) Lambda((n-k)/2) Lambda((n+k)/2)     0 < k <= n, k+n even,
 * and 0 otherwise.  Lambda is tabulated at half-integers by Lambda(0) = sqrt(pi),
 * Lambda(1/2) = 2/sqrt(pi), Lambda(z+1) = Lambda(z)(z+1/2)/(z+1).  It is pinned
 * by P_n(x) = sum_k M_{kn} T_k(x) (Eq. 14 context) in the tests.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (contraction must stay
 * off: the error-free transformations rely on separately rounded products).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* double-double arithmetic                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  double hi, lo;
} dd;

static inline dd dd_make(double hi, double lo) {
  dd r;
  r.hi = hi;
  r.lo = lo;
  return r;
}
static inline dd dd_from(double a) { return dd_make(a, 0.0); }

/* Knuth TwoSum: s + e == a + b exactly. */
static inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd_make(s, e);
}
/* Fast TwoSum, valid when |a| >= |b|. */
static inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  return dd_make(s, e);
}
/* TwoProd via fma: p + e == a * b exactly. */
static inline dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd_make(p, e);
}
static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static inline dd dd_neg(dd a) { return dd_make(-a.hi, -a.lo); }
static inline dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_add_d(dd a, double b) {
  dd s = two_sum(a.hi, b);
  s.lo += a.lo;
  return quick_two_sum(s.hi, s.lo);
}
/* Long division: three quotient digits, each corrected against the residual. */
static inline dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_mul_d(b, q1));
  double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_mul_d(b, q2));
  double q3 = r.hi / b.hi;
  dd q = quick_two_sum(q1, q2);
  return dd_add_d(q, q3);
}
static inline dd dd_div_d(dd a, double b) { return dd_div(a, dd_from(b)); }
/* Square root: one Newton step on the double estimate, carried out in dd. */
static inline dd dd_sqrt(dd a) {
  if (a.hi <= 0.0) return dd_from(0.0);
  double s = sqrt(a.hi);
  dd r = dd_sub(a, two_prod(s, s));
  return dd_add_d(dd_from(s), r.hi / (2.0 * s));
}
static inline double dd_abs_hi(dd a) { return fabs(a.hi); }

/* pi to double-double precision (the correctly rounded double and the
 * correctly rounded remainder). */
static const double PI_HI = 3.141592653589793116e+00;
static const double PI_LO = 1.224646799147353207e-16;

static inline dd dd_pi(void) { return dd_make(PI_HI, PI_LO); }

/* ------------------------------------------------------------------------ */
/* cos / sin of a dd angle in [-pi, 2pi]                                    */
/* ------------------------------------------------------------------------ */
/* Taylor series of sin and cos about 0 for |r| <= pi/4, summed in dd until the
 * term falls below 1e-36. */
static void dd_sincos_small(dd r, dd* s, dd* c) {
  dd r2 = dd_mul(r, r);
  dd term = r; /* r^(2j+1)/(2j+1)! */
  dd sum = r;
  for (int j = 1; j < 40; ++j) {
    term = dd_mul(term, r2);
    term = dd_div_d(term, (double)((2 * j) * (2 * j + 1)));
    term = dd_neg(term);
    sum = dd_add(sum, term);
    if (fabs(term.hi) < 1e-36) break;
  }
  *s = sum;
  term = dd_from(1.0); /* r^(2j)/(2j)! */
  sum = dd_from(1.0);
  for (int j = 1; j < 40; ++j) {
    term = dd_mul(term, r2);
    term = dd_div_d(term, (double)((2 * j - 1) * (2 * j)));
    term = dd_neg(term);
    sum = dd_add(sum, term);
    if (fabs(term.hi) < 1e-36) break;
  }
  *c = sum;
}

/* cos and sin of a dd angle: reduce by the nearest multiple j of pi/2, then
 * rotate the small-angle values by j quarter turns. */
void orc_sincos_dd(double th_hi, double th_lo, double* s_hi, double* s_lo,
                   double* c_hi, double* c_lo) {
  dd th = dd_make(th_hi, th_lo);
  dd half_pi = dd_mul_d(dd_pi(), 0.5);
  double jq = nearbyint(th.hi / half_pi.hi);
  int j = (int)jq;
  dd r = dd_sub(th, dd_mul_d(half_pi, jq));
  dd s, c;
  dd_sincos_small(r, &s, &c);
  int q = ((j % 4) + 4) % 4;
  dd so, co;
  switch (q) {
    case 0: so = s; co = c; break;
    case 1: so = c; co = dd_neg(s); break;
    case 2: so = dd_neg(s); co = dd_neg(c); break;
    default: so = dd_neg(c); co = s; break;
  }
  *s_hi = so.hi;
  *s_lo = so.lo;
  *c_hi = co.hi;
  *c_lo = co.lo;
}

/* ------------------------------------------------------------------------ */
/* Legendre polynomials by the three-term recurrence (dd)                   */
/* ------------------------------------------------------------------------ */
/* Coefficients of the recurrence (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1},
 * written as P_{m+1} = alpha_m x P_m - beta_m P_{m-1} with
 * alpha_m = (2m+1)/(m+1) and beta_m = m/(m+1) in dd, for m < n: entry 2m is
 * alpha_m, entry 2m+1 is beta_m.  Tabulating them once per call replaces a dd
 * division per step by two dd products (the same recurrence; results agree to
 * the dd rounding).  The caller frees the table. */
static dd* rec_coef(int64_t n) {
  dd* t = (dd*)malloc(sizeof(dd) * (size_t)(2 * (n > 0 ? n : 1)));
#pragma omp parallel for schedule(static)
  for (int64_t m = 0; m < n; ++m) {
    t[2 * m] = dd_div_d(dd_from((double)(2 * m + 1)), (double)(m + 1));
    t[2 * m + 1] = dd_div_d(dd_from((double)m), (double)(m + 1));
  }
  return t;
}

/* One step of the recurrence: P_{m+1} from P_m and P_{m-1}. */
static inline dd rec_step(const dd* coef, int64_t m, dd x, dd p, dd pm1) {
  return dd_sub(dd_mul(dd_mul(x, p), coef[2 * m]), dd_mul(pm1, coef[2 * m + 1]));
}

/* Returns P_n(x) and P_{n-1}(x) (P_{-1} := 0) by the recurrence above; coef
 * holds at least n coefficient pairs. */
static void legendre_pair_dd(int64_t n, dd x, const dd* coef, dd* pn, dd* pnm1) {
  dd pm1 = dd_from(0.0);
  dd p = dd_from(1.0);
  for (int64_t m = 0; m < n; ++m) {
    dd next = rec_step(coef, m, x, p, pm1);
    pm1 = p;
    p = next;
  }
  *pn = p;
  *pnm1 = pm1;
}

/* P_n at m double points (dd recurrence, rounded). */
void orc_legendre_p(int64_t n, const double* x, int64_t m, double* out) {
  dd* coef = rec_coef(n);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    dd pn, pnm1;
    legendre_pair_dd(n, dd_from(x[i]), coef, &pn, &pnm1);
    out[i] = pn.hi + pn.lo;
  }
  free(coef);
}

/* P_n at m dd points (x_hi + x_lo, e.g. the oracle's own nodes), rounded. */
void orc_legendre_p_dd(int64_t n, const double* x_hi, const double* x_lo, int64_t m, double* out) {
  dd* coef = rec_coef(n);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    dd pn, pnm1;
    legendre_pair_dd(n, dd_make(x_hi[i], x_lo[i]), coef, &pn, &pnm1);
    out[i] = pn.hi + pn.lo;
  }
  free(coef);
}

/* Chebyshev T_n at m double points by T_{j+1} = 2x T_j - T_{j-1} (dd). */
void orc_chebyshev_t(int64_t n, const double* x, int64_t m, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    dd xx = dd_from(x[i]);
    dd tm1 = dd_from(1.0), t = xx;
    if (n == 0) {
      out[i] = 1.0;
      continue;
    }
    for (int64_t j = 1; j < n; ++j) {
      dd next = dd_sub(dd_mul_d(dd_mul(xx, t), 2.0), tm1);
      tm1 = t;
      t = next;
    }
    out[i] = t.hi + t.lo;
  }
}

/* ------------------------------------------------------------------------ */
/* Legendre nodes and weights                                               */
/* ------------------------------------------------------------------------ */
/* Node k (0-based, theta ascending, i.e. x descending) of the N-point
 * Gauss-Legendre rule.  Newton's method on P_N(cos theta) in theta, started at
 * theta = (k+3/4)pi/(N+1/2) (the cheb* point, Sec. 2.2).  The derivative is
 * dP_N/dtheta = -N (P_{N-1}(x) - x P_N(x)) / sin(theta), from
 * (1-x^2) P_N'(x) = N (P_{N-1}(x) - x P_N(x)).  Three double-precision
 * iterations bring theta to about 1e-16; then dd iterations polish it until the
 * correction is below 1e-20 relative (quadratic convergence: the iterate is then
 * accurate to the dd rounding floor of the recurrence; near x = +-1 that floor is
 * about 1e-22 relative in theta at N = 2^20, because 1 - x carries the rounding
 * of cos(theta)).  The weight is 2/(dP_N/dtheta)^2 evaluated
 * at the final theta.  Returns the number of dd iterations used, or -1 when the
 * iteration did not settle. */
static int legpts_one(int64_t N, int64_t k, const dd* coef, dd* theta_out, dd* x_out, dd* w_out) {
  double th = ((double)k + 0.75) * M_PI / ((double)N + 0.5);
  /* double-precision Newton (the recurrence in double) */
  for (int it = 0; it < 3; ++it) {
    double x = cos(th), s = sin(th);
    double pm1 = 0.0, p = 1.0;
    for (int64_t m = 0; m < N; ++m) {
      double nx = ((double)(2 * m + 1) * x * p - (double)m * pm1) / (double)(m + 1);
      pm1 = p;
      p = nx;
    }
    double dp = -(double)N * (pm1 - x * p) / s;
    th -= p / dp;
  }
  dd t = dd_from(th);
  int used = -1;
  for (int it = 0; it < 8; ++it) {
    double sh, sl, ch, cl;
    orc_sincos_dd(t.hi, t.lo, &sh, &sl, &ch, &cl);
    dd s = dd_make(sh, sl), x = dd_make(ch, cl);
    dd pn, pnm1;
    legendre_pair_dd(N, x, coef, &pn, &pnm1);
    dd dp = dd_div(dd_mul_d(dd_sub(pnm1, dd_mul(x, pn)), -(double)N), s);
    dd delta = dd_div(pn, dp);
    t = dd_sub(t, delta);
    if (fabs(delta.hi) <= 1e-20 * fabs(t.hi)) {
      used = it + 1;
      break;
    }
  }
  /* weight and x at the final theta */
  double sh, sl, ch, cl;
  orc_sincos_dd(t.hi, t.lo, &sh, &sl, &ch, &cl);
  dd s = dd_make(sh, sl), x = dd_make(ch, cl);
  dd pn, pnm1;
  legendre_pair_dd(N, x, coef, &pn, &pnm1);
  dd dp = dd_div(dd_mul_d(dd_sub(pnm1, dd_mul(x, pn)), -(double)N), s);
  *w_out = dd_div(dd_from(2.0), dd_mul(dp, dp));
  *theta_out = t;
  *x_out = x;
  return used;
}

/* Nodes for the listed indices ks[0..nk).  Outputs (any may be NULL):
 * theta (hi, lo), x (hi, lo), w (hi, lo), and dtheta = theta_k - (k+1/2)pi/N
 * rounded to double (the offset from the cheb1 grid, Eq. 5 and Sec. 2.2).
 * Returns the number of nodes whose Newton iteration did not settle. */
int64_t orc_legpts(int64_t N, const int64_t* ks, int64_t nk, double* th_hi,
                   double* th_lo, double* x_hi, double* x_lo, double* w_hi,
                   double* w_lo, double* dtheta) {
  int64_t bad = 0;
  dd* coef = rec_coef(N);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (int64_t i = 0; i < nk; ++i) {
    dd th, x, w;
    int used = legpts_one(N, ks[i], coef, &th, &x, &w);
    if (used < 0) bad += 1;
    if (th_hi) th_hi[i] = th.hi;
    if (th_lo) th_lo[i] = th.lo;
    if (x_hi) x_hi[i] = x.hi;
    if (x_lo) x_lo[i] = x.lo;
    if (w_hi) w_hi[i] = w.hi;
    if (w_lo) w_lo[i] = w.lo;
    if (dtheta) {
      dd c1 = dd_div_d(dd_mul_d(dd_pi(), (double)ks[i] + 0.5), (double)N);
      dd d = dd_sub(th, c1);
      dtheta[i] = d.hi + d.lo;
    }
  }
  free(coef);
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Direct transforms                                                        */
/* ------------------------------------------------------------------------ */
/* Eq. 1 at selected rows: f_i = sum_{n<N} c_n P_n(x_i) with x_i given in dd. */
void orc_dlt_rows(int64_t N, const double* c, int64_t nk, const double* x_hi,
                  const double* x_lo, double* f) {
  dd* coef = rec_coef(N);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < nk; ++i) {
    dd x = dd_make(x_hi[i], x_lo[i]);
    dd pm1 = dd_from(0.0), p = dd_from(1.0);
    dd acc = dd_from(0.0);
    for (int64_t m = 0; m < N; ++m) {
      acc = dd_add(acc, dd_mul_d(p, c[m]));
      dd next = rec_step(coef, m, x, p, pm1);
      pm1 = p;
      p = next;
    }
    f[i] = acc.hi + acc.lo;
  }
  free(coef);
}

/* Transposed sums over a list of nodes (Sec. 4 matrix form):
 * out_n = s_n sum_{i<nk} g_i w_i P_n(x_i) for n < N, with x_i (and the optional
 * weights w_i; NULL = 1) in dd and s_n = n + 1/2 when scale_s is nonzero, else 1.
 * Over all N nodes with weights and the scale it is the IDLT, Eq. 2; without
 * them it is P^T g; over a subset of nodes it is the contribution of those rows
 * (equivalently, the transform of an input that vanishes off them).  Each
 * thread sums its rows into a private dd vector; the vectors are added in
 * thread order at the end. */
static void rows_t_impl(int64_t N, const double* g, int64_t nk, const double* x_hi, const double* x_lo,
                        const double* w_hi, const double* w_lo, int scale_s, double* out) {
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  dd* coef = rec_coef(N);
  dd* acc = (dd*)calloc((size_t)nthr * (size_t)N, sizeof(dd));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    dd* my = acc + (size_t)tid * (size_t)N;
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < nk; ++i) {
      dd x = dd_make(x_hi[i], x_lo[i]);
      dd gk = dd_from(g[i]);
      if (w_hi) gk = dd_mul(gk, dd_make(w_hi[i], w_lo ? w_lo[i] : 0.0));
      dd pm1 = dd_from(0.0), p = dd_from(1.0);
      for (int64_t m = 0; m < N; ++m) {
        my[m] = dd_add(my[m], dd_mul(p, gk));
        dd next = rec_step(coef, m, x, p, pm1);
        pm1 = p;
        p = next;
      }
    }
  }
  for (int64_t m = 0; m < N; ++m) {
    dd s = dd_from(0.0);
    for (int t = 0; t < nthr; ++t) s = dd_add(s, acc[(size_t)t * (size_t)N + m]);
    if (scale_s) s = dd_mul_d(s, (double)m + 0.5);
    out[m] = s.hi + s.lo;
  }
  free(acc);
  free(coef);
}

/* (P^T g)_n = sum_k g_k P_n(x_k) over all N nodes. */
void orc_dlt_t(int64_t N, const double* g, const double* x_hi, const double* x_lo,
               double* out) {
  rows_t_impl(N, g, N, x_hi, x_lo, NULL, NULL, 0, out);
}

/* The same over the listed nodes only: out_n = sum_{i<nk} g_i P_n(x_i), i.e.
 * P^T of an input that is zero off those rows. */
void orc_dlt_t_rows(int64_t N, const double* g, int64_t nk, const double* x_hi, const double* x_lo,
                    double* out) {
  rows_t_impl(N, g, nk, x_hi, x_lo, NULL, NULL, 0, out);
}

/* Contribution of a subset of rows to Eq. 2: out_n = (n+1/2) sum_{i<nk} w_i f_i
 * P_n(x_i) for the listed nodes (x_i, w_i in dd).  Summing it over a partition
 * of all N rows gives the IDLT. */
void orc_idlt_rows(int64_t N, const double* f, int64_t nk, const double* x_hi,
                   const double* x_lo, const double* w_hi, const double* w_lo, double* out) {
  rows_t_impl(N, f, nk, x_hi, x_lo, w_hi, w_lo, 1, out);
}

/* Eq. 2: c_n = (n+1/2) sum_k w_k f_k P_n(x_k). */
void orc_idlt(int64_t N, const double* f, const double* x_hi, const double* x_lo,
              const double* w_hi, const double* w_lo, double* c) {
  rows_t_impl(N, f, N, x_hi, x_lo, w_hi, w_lo, 1, c);
}

/* Eq. 3 at selected rows: f_i = sum_n c_n T_n(x_i), Chebyshev recurrence
 * T_{n+1} = 2x T_n - T_{n-1} (Sec. 2.4). */
void orc_ndct_rows(int64_t N, const double* c, int64_t nk, const double* x_hi,
                   const double* x_lo, double* f) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < nk; ++i) {
    dd x = dd_make(x_hi[i], x_lo[i]);
    dd tm1 = dd_from(1.0), t = dd_from(1.0); /* T_{-1} unused at m = 0 */
    dd acc = dd_from(0.0);
    for (int64_t m = 0; m < N; ++m) {
      dd tm;
      if (m == 0) {
        tm = dd_from(1.0);
      } else if (m == 1) {
        tm = x;
      } else {
        tm = dd_sub(dd_mul_d(dd_mul(x, t), 2.0), tm1);
      }
      acc = dd_add(acc, dd_mul_d(tm, c[m]));
      if (m >= 1) tm1 = t;
      t = tm;
    }
    f[i] = acc.hi + acc.lo;
  }
}

/* (T^T g)_n = sum_{i<nk} g_i T_n(x_i) for n < N over the listed nodes (Sec. 4
 * item 2); over all N nodes it is the transposed NDCT. */
void orc_ndct_t_rows(int64_t N, const double* g, int64_t nk, const double* x_hi, const double* x_lo,
                     double* out) {
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  dd* acc = (dd*)calloc((size_t)nthr * (size_t)N, sizeof(dd));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    dd* my = acc + (size_t)tid * (size_t)N;
#pragma omp for schedule(dynamic, 1)
    for (int64_t k = 0; k < nk; ++k) {
      dd x = dd_make(x_hi[k], x_lo[k]);
      dd gk = dd_from(g[k]);
      dd tm1 = dd_from(1.0), t = dd_from(1.0);
      for (int64_t m = 0; m < N; ++m) {
        dd tm;
        if (m == 0) {
          tm = dd_from(1.0);
        } else if (m == 1) {
          tm = x;
        } else {
          tm = dd_sub(dd_mul_d(dd_mul(x, t), 2.0), tm1);
        }
        my[m] = dd_add(my[m], dd_mul(tm, gk));
        if (m >= 1) tm1 = t;
        t = tm;
      }
    }
  }
  for (int64_t m = 0; m < N; ++m) {
    dd s = dd_from(0.0);
    for (int t = 0; t < nthr; ++t) s = dd_add(s, acc[(size_t)t * (size_t)N + m]);
    out[m] = s.hi + s.lo;
  }
  free(acc);
}

void orc_ndct_t(int64_t N, const double* g, const double* x_hi, const double* x_lo,
                double* out) {
  orc_ndct_t_rows(N, g, N, x_hi, x_lo, out);
}

/* ------------------------------------------------------------------------ */
/* Legendre -> Chebyshev coefficients: the matrix M of Sec. 3               */
/* ------------------------------------------------------------------------ */
/* lam[j] = Lambda(j/2) for j = 0..2N, Lambda(z) = Gamma(z+1/2)/Gamma(z+1). */
static dd* lambda_table(int64_t N) {
  dd* lam = (dd*)malloc((size_t)(2 * N + 2) * sizeof(dd));
  dd sqrt_pi = dd_sqrt(dd_pi());
  lam[0] = sqrt_pi;                               /* Gamma(1/2)/Gamma(1)   */
  lam[1] = dd_div(dd_from(2.0), sqrt_pi);         /* Gamma(1)/Gamma(3/2)   */
  for (int64_t j = 0; j + 2 <= 2 * N + 1; ++j) {  /* Lambda(z+1) = Lambda(z)(z+1/2)/(z+1) */
    lam[j + 2] = dd_div_d(dd_mul_d(lam[j], (double)(j + 1)), (double)(j + 2));
  }
  return lam;
}

/* Entry M_{kn} in dd (0 <= k, n < N). */
static dd m_entry(const dd* lam, int64_t k, int64_t n, dd inv_pi) {
  if (k > n || ((k + n) & 1)) return dd_from(0.0);
  if (k == 0) return dd_mul(inv_pi, dd_mul(lam[n], lam[n]));
  return dd_mul_d(dd_mul(inv_pi, dd_mul(lam[n - k], lam[n + k])), 2.0);
}

/* Dense entries of M (row-major [N][N]); for pinning M itself. */
void orc_leg2cheb_matrix(int64_t N, double* m) {
  dd* lam = lambda_table(N);
  dd inv_pi = dd_div(dd_from(1.0), dd_pi());
  for (int64_t k = 0; k < N; ++k)
    for (int64_t n = 0; n < N; ++n) {
      dd e = m_entry(lam, k, n, inv_pi);
      m[k * N + n] = e.hi + e.lo;
    }
  free(lam);
}

/* chat_k = sum_n M_{kn} c_n (Sec. 3, Eq. 14 context) for the listed k. */
void orc_leg2cheb_rows(int64_t N, const double* c, const int64_t* ks, int64_t nk, double* chat) {
  dd* lam = lambda_table(N);
  dd inv_pi = dd_div(dd_from(1.0), dd_pi());
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nk; ++i) {
    const int64_t k = ks[i];
    dd acc = dd_from(0.0);
    for (int64_t n = k; n < N; n += 2) acc = dd_add(acc, dd_mul_d(m_entry(lam, k, n, inv_pi), c[n]));
    chat[i] = acc.hi + acc.lo;
  }
  free(lam);
}

/* (M^T y)_n = sum_k M_{kn} y_k for the listed n. */
void orc_leg2cheb_t_rows(int64_t N, const double* y, const int64_t* ns, int64_t nn, double* out) {
  dd* lam = lambda_table(N);
  dd inv_pi = dd_div(dd_from(1.0), dd_pi());
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nn; ++i) {
    const int64_t n = ns[i];
    dd acc = dd_from(0.0);
    for (int64_t k = n & 1; k <= n; k += 2) acc = dd_add(acc, dd_mul_d(m_entry(lam, k, n, inv_pi), y[k]));
    out[i] = acc.hi + acc.lo;
  }
  free(lam);
}

/* chat = M c and out = M^T y over every index. */
void orc_leg2cheb(int64_t N, const double* c, double* chat) {
  int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) all[i] = i;
  orc_leg2cheb_rows(N, c, all, N, chat);
  free(all);
}

void orc_leg2cheb_t(int64_t N, const double* y, double* out) {
  int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  for (int64_t i = 0; i < N; ++i) all[i] = i;
  orc_leg2cheb_t_rows(N, y, all, N, out);
  free(all);
}

/* ------------------------------------------------------------------------ */
/* Plain FP64 direct method (the timed CPU baseline)                        */
/* ------------------------------------------------------------------------ */
/* P_N(x) and P_{N-1}(x) by (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1} in double. */
static void legendre_pair_f64(int64_t N, double x, double* pn, double* pnm1) {
  double pm1 = 0.0, p = 1.0;
  for (int64_t m = 0; m < N; ++m) {
    double next = ((double)(2 * m + 1) * x * p - (double)m * pm1) / (double)(m + 1);
    pm1 = p;
    p = next;
  }
  *pn = p;
  *pnm1 = pm1;
}

/* Nodes and weights in double: Newton in theta on P_N(cos theta) from the
 * cheb* point (k+3/4)pi/(N+1/2) (Sec. 2.2), derivative dP_N/dtheta =
 * -N (P_{N-1} - x P_N)/sin(theta).  Lemma 2.3 puts the start within
 * 1/(3 pi (2N+1)) of the root, about 1/60 of the node spacing ~pi/N, and Newton
 * converges quadratically from there (errors ~1e-2, 1e-4, 1e-8, 1e-16 of the
 * spacing), so five steps reach the rounding floor of the double recurrence
 * (near x = +-1 that floor is about N^2 u of the spacing).  A node whose fifth
 * step is still above 1e-6 of the spacing did not settle.  w = 2/(dP_N/dtheta)^2
 * at the final iterate.  Returns the number of nodes that did not settle. */
int64_t orc_legpts_f64(int64_t N, const int64_t* ks, int64_t nk, double* theta, double* x, double* w) {
  int64_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (int64_t i = 0; i < nk; ++i) {
    double th = ((double)ks[i] + 0.75) * M_PI / ((double)N + 0.5);
    double step = 0.0;
    for (int it = 0; it < 5; ++it) {
      double pn, pnm1;
      double c = cos(th), s = sin(th);
      legendre_pair_f64(N, c, &pn, &pnm1);
      double dp = -(double)N * (pnm1 - c * pn) / s;
      step = pn / dp;
      th -= step;
    }
    double pn, pnm1;
    double c = cos(th), s = sin(th);
    legendre_pair_f64(N, c, &pn, &pnm1);
    double dp = -(double)N * (pnm1 - c * pn) / s;
    if (!(fabs(step) * (double)N <= 1e-6)) bad += 1;
    if (theta) theta[i] = th;
    if (x) x[i] = c;
    if (w) w[i] = 2.0 / (dp * dp);
  }
  return bad;
}

/* Eq. 1 at the given rows, in double: f_i = sum_n c_n P_n(x_i). */
void orc_dlt_rows_f64(int64_t N, const double* c, int64_t nk, const double* x, double* f) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < nk; ++i) {
    double pm1 = 0.0, p = 1.0, acc = 0.0;
    for (int64_t m = 0; m < N; ++m) {
      acc += c[m] * p;
      double next = ((double)(2 * m + 1) * x[i] * p - (double)m * pm1) / (double)(m + 1);
      pm1 = p;
      p = next;
    }
    f[i] = acc;
  }
}

/* The given rows' contribution to Eq. 2, in double:
 * out_n = (n+1/2) sum_i w_i f_i P_n(x_i).  Each thread sums its rows into its
 * own length-N vector; the vectors are added at the end. */
void orc_idlt_rows_f64(int64_t N, const double* f, int64_t nk, const double* x, const double* w, double* out) {
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  double* acc = (double*)calloc((size_t)nthr * (size_t)N, sizeof(double));
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* my = acc + (size_t)tid * (size_t)N;
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < nk; ++i) {
      double g = w[i] * f[i];
      double pm1 = 0.0, p = 1.0;
      for (int64_t m = 0; m < N; ++m) {
        my[m] += g * p;
        double next = ((double)(2 * m + 1) * x[i] * p - (double)m * pm1) / (double)(m + 1);
        pm1 = p;
        p = next;
      }
    }
  }
  for (int64_t m = 0; m < N; ++m) {
    double s = 0.0;
    for (int t = 0; t < nthr; ++t) s += acc[(size_t)t * (size_t)N + m];
    out[m] = s * ((double)m + 0.5);
  }
  free(acc);
}

/* ------------------------------------------------------------------------ */
/* dd arithmetic self-checks exposed for the tests                          */
/* ------------------------------------------------------------------------ */
/* Returns (a*b) as (hi, lo) through TwoProd and (a+b) through TwoSum, so the
 * tests can confirm both are exact with integer arithmetic on the bits. */
void orc_two_prod(double a, double b, double* hi, double* lo) {
  dd r = two_prod(a, b);
  *hi = r.hi;
  *lo = r.lo;
}
void orc_two_sum(double a, double b, double* hi, double* lo) {
  dd r = two_sum(a, b);
  *hi = r.hi;
  *lo = r.lo;
}
void orc_dd_div(double ah, double al, double bh, double bl, double* qh, double* ql) {
  dd q = dd_div(dd_make(ah, al), dd_make(bh, bl));
  *qh = q.hi;
  *ql = q.lo;
}
void orc_dd_sqrt(double ah, double al, double* rh, double* rl) {
  dd r = dd_sqrt(dd_make(ah, al));
  *rh = r.hi;
  *rl = r.lo;
}
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
