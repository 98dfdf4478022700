// Plan creation, parameter derivation and the C-ABI entry points.
//
// Parameters (Sec. 2.2 Corollary 2.4 / Table 1; Sec. 3 "parameters determined
// by analysis for any working tolerance"):
//  * L (Taylor terms): the smallest L with 0.83845^L / L! <= eps/2.
//  * Asymptotic expansion of P_n(cos theta) with M terms and error bound
//    |R_M| <= 2 C_n h_{M,n} / (2 sin theta)^{M+1/2}: row theta_k may use it for
//    columns n >= n_cut(k) where the bound is <= eps/20.  Rows are grouped into
//    bands sharing one column cut; rows whose cut would exceed N use the
//    recurrence for every column.  M and the band cuts (from a geometric grid
//    of candidate cuts, ratio 2^(1/4)) minimise a cost model: each band costs M
//    FFTs of length N, each recurrence step a fixed cost per half row.
#include <algorithm>
#include <functional>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>

#include "gbdlt_internal.cuh"

namespace gbdlt {

static std::atomic<uint64_t> g_launches{0};
static std::atomic<uint64_t> g_allocs{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
cudaError_t dev_malloc(void** p, size_t bytes) {
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  return cudaMalloc(p, bytes);
}
static uint64_t launches_now() { return g_launches.load(std::memory_order_relaxed); }
static void uncount_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
int check_launch() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GBDLT_OK : GBDLT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// per-kernel profiler: one event after every launch; the interval between two
// consecutive events is the device time of the kernel launched between them
// (kernels on one stream run back to back)
// ---------------------------------------------------------------------------
struct ProfMark {
  const char* name;
  double flops, bytes;
};
struct ProfAcc {
  int64_t count = 0;
  double ms = 0, flops = 0, bytes = 0;
};
struct Profiler {
  bool on = false;
  bool anchored = false;
  std::vector<cudaEvent_t> ev;  // ev[0] anchor; ev[i+1] recorded after marks[i]
  std::vector<ProfMark> marks;
  std::map<std::string, ProfAcc> acc;
};

static void prof_flush(Plan& P) {
  Profiler& R = *P.prof;
  const size_t n = R.marks.size();
  if (n == 0) return;
  cudaEventSynchronize(R.ev[n]);
  for (size_t i = 0; i < n; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, R.ev[i], R.ev[i + 1]);
    ProfAcc& a = R.acc[R.marks[i].name];
    a.count += 1;
    a.ms += ms;
    a.flops += R.marks[i].flops;
    a.bytes += R.marks[i].bytes;
  }
  std::swap(R.ev[0], R.ev[n]);
  R.marks.clear();
}

void launched(Plan& P, const char* name, double flops, double bytes) {
  count_launch();
  if (!P.prof || !P.prof->on || !P.prof->anchored) return;
  Profiler& R = *P.prof;
  if (R.marks.size() + 1 >= R.ev.size()) prof_flush(P);
  cudaEventRecord(R.ev[R.marks.size() + 1], P.stream);
  R.marks.push_back(ProfMark{name, flops, bytes});
}

// ---------------------------------------------------------------------------
// host double-double (for the C_n table)
// ---------------------------------------------------------------------------
namespace {
struct hdd {
  double hi, lo;
};
hdd h_quick(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
hdd h_two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
hdd h_mul_d(hdd a, double b) {
  hdd p = h_two_prod(a.hi, b);
  p.lo = std::fma(a.lo, b, p.lo);
  return h_quick(p.hi, p.lo);
}
hdd h_div_d(hdd a, double b) {
  double q1 = a.hi / b;
  hdd p = h_two_prod(q1, b);
  double r = ((a.hi - p.hi) - p.lo) + a.lo;
  double q2 = r / b;
  return h_quick(q1, q2);
}
}  // namespace

std::vector<double> cn_table(int64_t N) {
  // C_0 = 4/pi; C_{n+1} = C_n (n+1)/(n+3/2)
  std::vector<double> C((size_t)N + 1);
  hdd c = {1.2732395447351628, -7.871470670072994e-17};  // 4/pi to double-double
  for (int64_t n = 0; n <= N; ++n) {
    C[(size_t)n] = c.hi + c.lo;
    c = h_div_d(h_mul_d(c, (double)(n + 1)), (double)n + 1.5);
  }
  return C;
}

static std::vector<double> head_table(int64_t h) {
  // Lam'_0 = sqrt(2/pi) Gamma(1/2) = sqrt(2); Lam'_{j+1} = Lam'_j (j+1/2)/(j+1)
  std::vector<double> L((size_t)h);
  hdd v = {1.4142135623730951, -9.667293313452913e-17};  // sqrt(2) to double-double
  for (int64_t j = 0; j < h; ++j) {
    L[(size_t)j] = v.hi + v.lo;
    v = h_div_d(h_mul_d(v, (double)j + 0.5), (double)(j + 1));
  }
  return L;
}

// ---------------------------------------------------------------------------
// parameter derivation
// ---------------------------------------------------------------------------
static double log_gM(int M, double n) {
  // log(2 C_n h_{M,n})
  double lc = 0.5 * std::log(4.0 / M_PI) + std::lgamma(n + 1.0) - std::lgamma(n + 1.5);
  double lh = 0.0;
  for (int j = 1; j <= M; ++j) lh += 2.0 * std::log(j - 0.5) - std::log((double)j) - std::log(n + j + 0.5);
  return std::log(2.0) + lc + lh;
}

struct DPResult {
  double cost = 0;
  std::vector<Band> bands;
};

// first half row k (theta_k = (k+1/2) pi/N) at which the M-term remainder bound
// of columns n >= ns is below eps_asy, or H when none is
static int64_t first_row(int64_t N, int M, double eps_asy, int64_t ns) {
  const int64_t H = N / 2;
  double lgm = log_gM(M, (double)ns);
  double lsmin = (lgm - std::log(eps_asy)) / (M + 0.5) - std::log(2.0);
  double smin = std::exp(lsmin);
  if (smin >= 1.0) return H;
  double kk = (double)N * std::asin(smin) / M_PI - 0.5;
  int64_t k = (int64_t)std::ceil(kk);
  if (k < 0) k = 0;
  // guard against rounding of asin: move to the first row that satisfies the bound
  while (k < H && std::sin((k + 0.5) * M_PI / N) < smin) ++k;
  while (k > 0 && std::sin((k - 0.5) * M_PI / N) >= smin) --k;
  return std::min(k, H);
}

// FP64 plans: how many leading expansion terms of a band must have FP64 FFTs.
// At the band's first row, term m of columns n >= ns is at most
// T_m = 2 C_ns h_{m,ns} / (2 sin theta_ka)^{m+1/2} ||c||_1 (the remainder bound
// with m terms), and an FFT in FP32 of its vector errs by at most about
// 2 log2(N) u_32 T_m; the terms run in FP32 are the tail m >= Mh whose errors
// sum to at most eps/20.
// unit: the relative error per operation of the cheaper arithmetic (2^-24 for
// FP32; 2^-46 for float-float, two bits above its significand for the cheap
// additions).
static int fp64_terms(int64_t N, int M, double eps, int64_t ns, int64_t ka, double unit = 0x1p-24) {
  int lg = 0;
  while ((1ll << lg) < N) ++lg;
  const double s2 = 2.0 * std::sin(((double)ka + 0.5) * M_PI / (double)N);
  const double ferr = 2.0 * std::max(lg, 1) * unit;
  double err = 0.0;
  int Mh = M;
  while (Mh > 1) {
    const double Tm = std::exp(log_gM(Mh - 1, (double)ns) - (Mh - 0.5) * std::log(s2));
    if (err + ferr * Tm > eps / 20.0) break;
    err += ferr * Tm;
    --Mh;
  }
  return Mh;
}

// tcost: the FFTs of one band (all its terms); prune_kb: a band whose rows end at
// kb <= prune_kb has its FFTs pruned to two windows of bins (fft.cu), costing
// about prune_f of a full band's FFTs.
// head: columns n < head come from the dense head block M[0:head, 0:head]
// (head.cu), so no band cuts below it and every row's recurrence starts there.
static DPResult plan_bands(int64_t N, int M, double eps_asy, double tcost, double c_rec, int64_t prune_kb,
                           double prune_f, int64_t head) {
  const int64_t H = N / 2;
  DPResult best_res;
  // candidate cuts, descending (none below the head; the head itself is one)
  std::vector<int64_t> cands;
  int lg = 0;
  while ((1ll << lg) < N) ++lg;
  for (int i = 4 * lg; i >= 4; --i) {
    int64_t v = (int64_t)std::llround(std::pow(2.0, i / 4.0));
    v = std::min<int64_t>(v, N);
    if (head > 0 && v < head) break;
    if (v >= 2 && (cands.empty() || cands.back() != v)) cands.push_back(v);
  }
  if (head > 0 && (cands.empty() || cands.back() != head)) cands.push_back(head);
  const int nc = (int)cands.size();
  // first half row whose n_cut <= cand
  std::vector<int64_t> Kc(nc);
  for (int i = 0; i < nc; ++i) Kc[i] = first_row(N, M, eps_asy, cands[i]);
  std::vector<double> best(nc, 0.0);
  std::vector<int> choice(nc, -1);
  for (int i = nc - 1; i >= 0; --i) {
    const int64_t ka = Kc[i];
    if (ka >= H) {
      best[i] = 0.0;
      choice[i] = -2;  // empty
      continue;
    }
    const double rows_rec = (double)(cands[i] - head) * c_rec;  // per row of the band
    double opt = tcost + rows_rec * (double)(H - ka);
    int ch = -1;
    for (int j = i + 1; j < nc; ++j) {
      const int64_t kb = Kc[j];
      if (kb <= ka) continue;
      const double bt = kb <= prune_kb ? prune_f * tcost : tcost;
      double c2 = bt + rows_rec * (double)(kb - ka) + best[j];
      if (c2 < opt) {
        opt = c2;
        ch = j;
      }
    }
    best[i] = opt;
    choice[i] = ch;
  }
  const double full_rec = (double)(N - head) * c_rec;  // per row below the first band
  double top = full_rec * (double)H;
  int topi = -1;
  for (int i = 0; i < nc; ++i) {
    if (choice[i] == -2) continue;
    double c0 = full_rec * (double)Kc[i] + best[i];
    if (c0 < top) {
      top = c0;
      topi = i;
    }
  }
  best_res.cost = top;
  int i = topi;
  while (i >= 0) {
    const int j = choice[i];
    const int64_t ka = Kc[i];
    const int64_t kb = j >= 0 ? Kc[j] : H;
    if (kb > ka) best_res.bands.push_back(Band{cands[i], ka, kb});
    i = j;
  }
  return best_res;
}

int derive_params(int64_t N, int prec, double eps, int method, Params* p, double taylor_b) {
  if (N < 1 || N > (1ll << 24)) return GBDLT_ERR_UNSUPPORTED_N;
  if (prec != GBDLT_FP64 && prec != GBDLT_FP32) return GBDLT_ERR_INVALID_ARG;
  if (method != GBDLT_METHOD_AUTO && method != GBDLT_METHOD_FAST && method != GBDLT_METHOD_DIRECT)
    return GBDLT_ERR_INVALID_ARG;
  if (eps <= 0.0) eps = prec == GBDLT_FP64 ? 1e-14 : 2e-6;
  if (!(eps < 1.0) || !std::isfinite(eps)) return GBDLT_ERR_INVALID_ARG;
  const bool pow2 = (N & (N - 1)) == 0;
  if (method == GBDLT_METHOD_AUTO) method = N <= kDirectAuto ? GBDLT_METHOD_DIRECT : GBDLT_METHOD_FAST;
  if (method == GBDLT_METHOD_DIRECT && N > kDirectMax) return GBDLT_ERR_UNSUPPORTED_N;
  if (method == GBDLT_METHOD_FAST && !pow2) {
    // The chain on the power-of-two grid G > N (FFT length G): the coefficients
    // are zero-padded to G (leg2cheb of the padded vector gives the same
    // Chebyshev coefficients: the Legendre series has degree N - 1 < G) and every
    // row theta_k of the N-point rule takes its Taylor expansion about the
    // nearest point (j + 1/2) pi / G of the grid, |theta_k - theta'_j| <= pi/(2G).
    // Over the columns n < N, |n dtheta_k| <= (N - 1) pi / (2G): the bound of
    // Corollary 2.4 with that in place of 0.83845 fixes L.
    int64_t G = 1;
    while (G < N) G <<= 1;
    const double b = (double)(N - 1) * M_PI / (2.0 * (double)G) * (1.0 + 1e-9);
    Params q;
    int st = derive_params(G, prec, eps, GBDLT_METHOD_FAST, &q, b);
    if (st) return st;
    q.N = N;
    q.direct_steps = N <= kDirectMax ? ((N + 1) / 2) * N : 0;
    const double dsz = prec == GBDLT_FP64 ? 8.0 : 4.0;
    q.bytes_dlt = (2.0 * dsz + 8.0) * (double)N;
    q.bytes_idlt = (2.0 * dsz + 16.0) * (double)N;
    *p = q;
    return GBDLT_OK;
  }
  Params q;
  q.N = N;
  q.prec = prec;
  q.eps = eps;
  q.method = method;
  q.fast = pow2;
  q.grid = pow2 ? N : 0;
  q.taylor_b = taylor_b;
  // Corollary 2.4 with theta* = theta^cheb1: |f - f_L| <= b^L / L! ||c||_1,
  // b = 0.83845 (or the bound of a grid plan's rows)
  int L = 1;
  double b = taylor_b;
  while (b > 0.5 * eps && L < 24) {
    ++L;
    b *= taylor_b / L;
  }
  q.L = L;
  // Taylor terms l >= Lff run their FFTs and combines in float-float in FP64
  // plans: term l is at most b^l / l! ||c||_1 (Corollary 2.4) and a
  // float-float FFT of it errs by about 2 log2(N) 2^-46 of that; the tail
  // l >= Lff keeps the sum of those errors within eps/20
  q.Lff = L;
  if (prec == GBDLT_FP64) {
    int lgN = 0;
    while ((1ll << lgN) < N) ++lgN;
    const double ferr = 2.0 * std::max(lgN, 1) * 0x1p-46;
    double err = 0.0;
    for (int l = L - 1; l >= 1; --l) {
      double tl = 1.0;
      for (int i = 1; i <= l; ++i) tl *= taylor_b / i;
      if (err + ferr * tl > eps / 20.0) break;
      err += ferr * tl;
      q.Lff = l;
    }
  }
  // recurrence segment length of the fast path's layout: 512 columns, 256 in
  // FP32 plans, whose shorter float-float recurrence kernels balance better over
  // the SMs in finer pieces (2^20: forward 0.105 -> 0.090 ms, transposed 0.121
  // -> 0.094 ms; FP64 plans measured the same either way)
  q.seg = prec == GBDLT_FP32 ? 256 : 512;
  q.M = 0;
  q.K = 0;
  int lg = 0;
  while ((1ll << lg) < N) ++lg;
  if (pow2 && N >= 4) {
    const double eps_asy = eps / 20.0;
    // costs in picoseconds of GB300 time, fitted to the measured kernels at
    // N = 2^20: one FFT vector of the pipeline (forward and transposed chain)
    // per point, and one recurrence step of a half row (both directions averaged)
    // c_head: one term M_kn c_n of the dense head block (two FP64 instructions
    // in the FP64 form; FP32 arithmetic with a compensated sum in the FP32 form)
    // c_fft32: an FP32 FFT vector (the FP32 form's, and the FP32 tail terms of
    // an FP64 plan's bands); c_fftff: a float-float FFT vector (the mid terms)
    // (each with its term's share of the prologue/epilogue kernels)
    const double c_fft32 = (0.8 * lg + 10.0) * (double)N;  // memory and shared-memory bound FP32 passes
    const double c_fftff = (2.0 * lg + 13.0) * (double)N;  // FP32-pipe bound
    double c_fft, c_rec, c_head;
    int Mmax;
    if (prec == GBDLT_FP64) {
      c_fft = (4.33 * lg + 16.0) * (double)N;  // ~64 FP64 instructions per point at 2^20
      c_rec = 7.7;                             // ~4.8 FP64 instructions per step
      c_head = 4.0;
      Mmax = 24;
    } else {
      c_fft = (0.43 * lg + 1.7) * (double)N;  // the FP32 form's passes and combines
      c_rec = 3.4;                             // float-float recurrence
      c_head = 0.25;
      Mmax = 16;
    }
    double best = (double)N * c_rec * (double)(N / 2);  // all recurrence
    int64_t prune_kb = 0;
    if (N > 4096) {
      const int64_t L1 = 1ll << (lg / 2), L2 = N / L1;
      prune_kb = std::min(L1, L2) - 4;  // 2 (kb/2 + 2) <= min(L1, L2)
    }
    // head sizes: 0 or a power-of-two multiple of 512 (a multiple of the
    // segment length), at most N/4 and kHeadMax
    std::vector<int64_t> heads = {0};
    for (int64_t h = 512; h <= std::min<int64_t>(N / 4, kHeadMax); h *= 2) heads.push_back(h);
    for (int64_t h : heads) {
      const double head_cost = c_head * 0.25 * (double)h * (double)h;  // h^2/4 terms
      for (int M = 2; M <= Mmax; ++M) {
        // FP64 plans: the FP64 share of a band's terms, estimated on a band
        // with cut max(h, sqrt N) at its first row (the split is nearly the same
        // for every band: each starts where its own bound meets eps/20)
        int Mh = M, M64 = M;
        if (prec == GBDLT_FP64) {
          const int64_t ns_rep = std::max<int64_t>(h, 1ll << (lg / 2));
          const int64_t ka_rep = first_row(N, M, eps_asy, ns_rep);
          Mh = fp64_terms(N, M, eps, ns_rep, ka_rep);
          M64 = fp64_terms(N, Mh, eps, ns_rep, ka_rep, 0x1p-46);
        }
        const double tcost = (double)M64 * c_fft + (double)(Mh - M64) * c_fftff + (double)(M - Mh) * c_fft32;
        // pruned bands save FP64 work; the FP32 passes are bound by memory
        // latency, where the saving is small
        DPResult r = plan_bands(N, M, eps_asy, tcost, c_rec, prune_kb, prec == GBDLT_FP64 ? 0.6 : 1.0, h);
        if ((int)r.bands.size() > GBDLT_MAX_BANDS) continue;
        if (r.cost + head_cost < best) {
          best = r.cost + head_cost;
          q.M = M;
          q.bands = r.bands;
          q.head = h;
        }
      }
    }
    q.K = (int)q.bands.size();
    if (q.K == 0) q.M = 0;
    // the split of the chosen bands: every band's FP32 tail within its budget
    q.Mh = q.M;
    q.M64 = q.M;
    if (prec == GBDLT_FP64 && q.K > 0) {
      q.Mh = 1;
      for (const Band& bd : q.bands) q.Mh = std::max(q.Mh, fp64_terms(N, q.M, eps, bd.ns, bd.ka));
      q.M64 = 1;
      for (const Band& bd : q.bands) q.M64 = std::max(q.M64, fp64_terms(N, q.Mh, eps, bd.ns, bd.ka, 0x1p-46));
    }
  }
  // recurrence work of the fast path (cheb1 rows), and of the direct method
  // (every Legendre node row against every column, mirrored rows shared)
  const int64_t H = N / 2;
  int64_t half_steps = 0;
  if (pow2) {
    int64_t k0 = q.K > 0 ? q.bands[0].ka : H;
    half_steps += k0 * (N - q.head);
    for (const Band& bd : q.bands) half_steps += (bd.kb - bd.ka) * (bd.ns - q.head);
  }
  q.rec_steps = 2 * half_steps;
  q.direct_steps = N <= kDirectMax ? ((N + 1) / 2) * N : 0;
  const int npair = (q.L - 1 + 1) / 2;
  const double fft_flops = 5.0 * (double)N * (double)std::max(lg, 1);
  q.flops_dlt = method == GBDLT_METHOD_DIRECT
                    ? 7.0 * (double)q.direct_steps
                    : (double)(q.K * q.M + 1 + npair) * fft_flops + 7.0 * (double)half_steps +
                          0.5 * (double)q.head * (double)q.head;
  const double dsz = prec == GBDLT_FP64 ? 8.0 : 4.0;
  q.bytes_dlt = (2.0 * dsz + 8.0) * (double)N;
  q.bytes_idlt = (2.0 * dsz + 16.0) * (double)N;
  *p = q;
  return GBDLT_OK;
}

// ---------------------------------------------------------------------------
// tables on the device
// ---------------------------------------------------------------------------
namespace {
__global__ void k_twiddle(double2* out, int64_t count, int64_t B, int64_t mult) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t e = (i * mult) % B;
  double s, c;
  sincospi(2.0 * (double)e / (double)B, &s, &c);
  out[i] = make_double2(c, s);
}
void twiddle_fill(Plan& P, double2* out, int64_t count, int64_t B, int64_t mult) {
  k_twiddle<<<(unsigned)((count + 255) / 256), 256, 0, P.stream>>>(out, count, B, mult);
  count_launch();
}
__global__ void k_to_float2(const double2* in, float2* out, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
void to_float(Plan& P, const double2* in, float2* out, int64_t count) {
  k_to_float2<<<(unsigned)((count + 255) / 256), 256, 0, P.stream>>>(in, out, count);
  count_launch();
}
}  // namespace

int launch_twiddle_init(Plan& P) {
  twiddle_fill(P, P.tw4096, 4096, 4096, 1);
  twiddle_fill(P, P.twN.lo, 4096, P.twN.B, 1);
  twiddle_fill(P, P.twN.hi, std::max<int64_t>(1, P.twN.B / 4096), P.twN.B, 4096);
  twiddle_fill(P, P.tw4N.lo, 4096, P.tw4N.B, 1);
  twiddle_fill(P, P.tw4N.hi, std::max<int64_t>(1, P.tw4N.B / 4096), P.tw4N.B, 4096);
  if (P.twfull) twiddle_fill(P, P.twfull, P.p.N, P.p.N, 1);
  to_float(P, P.tw4096, P.tw4096f, 4096);
  to_float(P, P.twN.lo, P.twNf_lo, 4096);
  to_float(P, P.twN.hi, P.twNf_hi, std::max<int64_t>(1, P.twN.B / 4096));
  to_float(P, P.tw4N.lo, P.tw4Nf_lo, 4096);
  to_float(P, P.tw4N.hi, P.tw4Nf_hi, std::max<int64_t>(1, P.tw4N.B / 4096));
  return check_launch();
}

// ---------------------------------------------------------------------------
// plan lifecycle
// ---------------------------------------------------------------------------
namespace {

struct Arena {
  size_t off = 0;
  template <typename U>
  size_t take(int64_t count) {
    size_t o = off;
    off += ((size_t)std::max<int64_t>(count, 1) * sizeof(U) + 255) & ~(size_t)255;
    return o;
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// Graph replay of transform chains.  A chain is 10-60 kernel launches; for small
// N their launch latency is most of a call.  The third and later calls with the
// same (operator, method, pointers, batch) replay a CUDA graph captured on the
// plan's internal stream (the first call runs the chain directly, which settles
// kernel attributes; the second captures and replays).  The internal stream
// waits for the caller's stream and the caller's stream for the replay, so the
// calls keep the caller's stream order.  Chains are not replayed while the
// per-kernel profiler is on or while the caller's stream is itself being
// captured (the caller's graph then records the kernels).
// ---------------------------------------------------------------------------
struct GraphEntry {
  int op = 0, method = 0;
  bool nodes = false;  // the chain runs the deferred node kernel
  const void* in = nullptr;
  void* out = nullptr;
  int64_t batch = 0;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;
  uint64_t last = 0;
  int calls = 0;
};
struct GraphCache {
  cudaStream_t s = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
  std::vector<GraphEntry> e;
  uint64_t tick = 0;
  bool broken = false;  // a capture failed: run chains directly from now on
};
constexpr size_t kGraphCacheSize = 16;

void free_graphs(Plan* P) {
  GraphCache* G = P->graphs;
  if (!G) return;
  for (GraphEntry& x : G->e)
    if (x.exec) cudaGraphExecDestroy(x.exec);
  if (G->in) cudaEventDestroy(G->in);
  if (G->out) cudaEventDestroy(G->out);
  if (G->s) cudaStreamDestroy(G->s);
  delete G;
  P->graphs = nullptr;
}

void free_plan(Plan* P) {
  if (!P) return;
  if (P->graphs) {
    cudaStreamSynchronize(P->graphs->s);
    free_graphs(P);
  }
  if (P->side) {
    cudaStreamSynchronize(P->side);
    cudaStreamDestroy(P->side);
  }
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  if (P->node_s) {
    cudaStreamSynchronize(P->node_s);
    cudaStreamDestroy(P->node_s);
  }
  if (P->node_fork) cudaEventDestroy(P->node_fork);
  if (P->node_join) cudaEventDestroy(P->node_join);
  if (P->arena) cudaFree(P->arena);
  if (P->inner) free_plan(P->inner);
  if (P->rg_in) cudaFree(P->rg_in);
  if (P->rg_g) cudaFree(P->rg_g);
  if (P->rg_own) grid_rules_free(P->rg_own);
  if (P->prof) {
    for (cudaEvent_t e : P->prof->ev) cudaEventDestroy(e);
    delete P->prof;
  }
  delete P;
}


namespace {

// Host side of a recurrence layout: rows [0, H) with column cuts `cut`, cut into
// segments of S columns; CTAs are (row block of 256 half rows, segment) pairs.
// Segments below j0 (the columns of the dense head block) are not run: a row
// stores its segments j0 .. nseg-1, and a row block's transposed partials cover
// columns [j0 S, nseg_max S).
struct LayoutHost {
  std::vector<int32_t> cut, cta_rb, cta_j, maxcut, fw_rb, fw_lane;
  std::vector<int32_t> tw_k, tw_slot, tslot_j, tseg_begin;
  std::vector<int64_t> poff, toff;
};

void build_ctas(RecLayout& R, int64_t H, int S, int j0, int pack, LayoutHost& h);

void layout_build(RecLayout& R, int64_t H, int S, std::vector<int32_t> cut, int j0, int sms, int64_t batch,
                  bool packed_t, LayoutHost& h) {
  R.H = H;
  R.S = S;
  R.j0 = j0;
  h.cut = std::move(cut);
  h.poff.assign((size_t)std::max<int64_t>(H, 1), 0);
  int64_t o = 0, steps = 0;
  R.n_long = 0;
  const int64_t n_lo = (int64_t)j0 * S;
  for (int64_t k = 0; k < H; ++k) {
    h.poff[(size_t)k] = o;
    const int64_t ns = std::max<int64_t>(0, (h.cut[(size_t)k] + S - 1) / S - j0);
    o += ns;
    steps += std::max<int64_t>(0, h.cut[(size_t)k] - n_lo);
    if (ns > 64) R.n_long = k + 1;
  }
  R.nseg_total = o;
  R.half_steps = steps;
  R.nblocks = (H + 255) / 256;
  // CTAs: segments of a row block, several per CTA when their active rows fill
  // only A < 8 warps (A warps per segment, q = 8 / A segments), provided the
  // packed launch still has two CTAs per SM over the batch the plan is made for
  // (small transforms need the SMs more than full CTAs; the per-segment
  // arithmetic is the same either way)
  for (int pack = 1; pack >= 0; --pack) {
    h.cta_rb.clear();
    h.cta_j.clear();
    h.maxcut.clear();
    h.toff.clear();
    build_ctas(R, H, S, j0, pack, h);
    if (!pack || (int64_t)h.cta_rb.size() * batch >= 2 * (int64_t)sms) break;
  }
  R.ncta = (int64_t)h.cta_rb.size();
  // the forward recurrence's warps: per row block the pairs (segment j >= j0,
  // row r) with r up to the last row whose cut reaches segment j, segment by
  // segment, 32 to a warp (a block's last warp padded with -1), so that a
  // segment whose active rows do not fill whole warps shares warps with the
  // next; CTAs of 2 warps (in CTAs of 8 the 857 CTAs at 2^20 fell 5 or 6 to an
  // SM and the SMs with 5 idled at the end: 0.811 -> 0.789 ms), 1 where that
  // would leave fewer than two CTAs per SM over the plan's batch
  h.fw_rb.clear();
  h.fw_lane.clear();
  std::vector<std::vector<int>> lastr_rb((size_t)R.nblocks);  // per row block, per segment: last row
  for (int64_t rb = 0; rb < R.nblocks; ++rb) {
    const int64_t r0 = rb * 256, r1 = std::min<int64_t>(H, rb * 256 + 256);
    int64_t nsm = 0;
    for (int64_t k = r0; k < r1; ++k) nsm = std::max<int64_t>(nsm, (h.cut[(size_t)k] + S - 1) / S);
    std::vector<int> lastr((size_t)std::max<int64_t>(nsm, 1), -1);
    for (int64_t k = r0; k < r1; ++k) {
      const int64_t ns = (h.cut[(size_t)k] + S - 1) / S;
      if (ns > 0) lastr[(size_t)ns - 1] = std::max(lastr[(size_t)ns - 1], (int)(k - r0));
    }
    for (int64_t j = nsm - 2; j >= 0; --j) lastr[(size_t)j] = std::max(lastr[(size_t)j], lastr[(size_t)j + 1]);
    const size_t first = h.fw_lane.size();
    for (int64_t j = j0; j < nsm; ++j)
      for (int r = 0; r <= lastr[(size_t)j]; ++r) h.fw_lane.push_back((int32_t)(r | (j << 8)));
    while ((h.fw_lane.size() - first) % 32) h.fw_lane.push_back(-1);
    for (size_t w = first / 32; w < h.fw_lane.size() / 32; ++w) h.fw_rb.push_back((int32_t)rb);
    if (nsm > j0) lastr_rb[(size_t)rb] = std::move(lastr);
  }
  // the transposed recurrence's warps (fast layouts): the pairs (half row k,
  // segment j) ordered by segment, then row block, then row, 32 to a warp; a
  // warp's lanes of one segment form a run, and every run has a slot of S
  // column sums (tpart), so that the slots of segment j are the contiguous range
  // tseg_begin[j - j0] .. tseg_begin[j - j0 + 1] (rec.cu, k_rec_tp)
  h.tw_k.clear();
  h.tw_slot.clear();
  h.tslot_j.clear();
  h.tseg_begin.clear();
  R.ntw = R.tslots = 0;
  R.tsegs = 0;
  if (packed_t) {
    std::vector<int64_t> act;  // row blocks that run segments
    int64_t jmax = j0;
    for (int64_t rb = 0; rb < R.nblocks; ++rb)
      if (!lastr_rb[(size_t)rb].empty()) {
        act.push_back(rb);
        jmax = std::max<int64_t>(jmax, (int64_t)lastr_rb[(size_t)rb].size());
      }
    int32_t slot = -1, last_j = -1;
    for (int64_t j = j0; j < jmax; ++j) {
      h.tseg_begin.push_back(slot + 1);
      for (int64_t rb : act) {
        const std::vector<int>& lr = lastr_rb[(size_t)rb];
        if (j >= (int64_t)lr.size()) continue;
        for (int r = 0; r <= lr[(size_t)j]; ++r) {
          if (h.tw_k.size() % 32 == 0 || last_j != (int32_t)j) {
            h.tslot_j.push_back((int32_t)j);
            ++slot;
          }
          last_j = (int32_t)j;
          h.tw_k.push_back((int32_t)(rb * 256 + r));
          h.tw_slot.push_back(slot);
        }
      }
    }
    h.tseg_begin.push_back(slot + 1);
    while (h.tw_k.size() % 32) {
      h.tw_k.push_back(-1);
      h.tw_slot.push_back(-1);
    }
    R.ntw = (int64_t)h.tw_k.size() / 32;
    R.tslots = (int64_t)h.tslot_j.size();
    R.tsegs = (int)(jmax - j0);
    R.twpc = 8;
    while (R.twpc > 1 && ((R.ntw + R.twpc - 1) / R.twpc) * batch < 2 * (int64_t)sms) R.twpc /= 2;
  }
  R.nfw = (int64_t)h.fw_rb.size();
  R.fwpc = 2;
  while (R.fwpc > 1 && ((R.nfw + R.fwpc - 1) / R.fwpc) * batch < 2 * (int64_t)sms) R.fwpc /= 2;
  // the transposed reduction relies on row blocks in order of non-increasing cut
  // (true by construction: full rows first, then bands of decreasing cut)
  std::vector<int32_t> mc = h.maxcut;
  std::sort(mc.begin(), mc.end(), std::greater<int32_t>());
  R.n_heavy = mc.size() > 32 ? mc[32] : 0;
}

void build_ctas(RecLayout& R, int64_t H, int S, int j0, int pack, LayoutHost& h) {
  int64_t to = 0;
  std::vector<int> lastr;  // per segment: last row of the block that runs it
  for (int64_t rb = 0; rb < R.nblocks; ++rb) {
    const int64_t r0 = rb * 256, r1 = std::min<int64_t>(H, rb * 256 + 256);
    int32_t mc = 0;
    for (int64_t k = r0; k < r1; ++k) mc = std::max(mc, h.cut[(size_t)k]);
    const int64_t nsm = (mc + S - 1) / S;
    h.maxcut.push_back(mc);
    h.toff.push_back(to);
    to += std::max<int64_t>(0, nsm - j0) * S;
    lastr.assign((size_t)std::max<int64_t>(nsm, 1), -1);
    for (int64_t k = r0; k < r1; ++k) {
      const int64_t ns = (h.cut[(size_t)k] + S - 1) / S;
      if (ns > 0) lastr[(size_t)ns - 1] = std::max(lastr[(size_t)ns - 1], (int)(k - r0));
    }
    for (int64_t j = nsm - 2; j >= 0; --j) lastr[(size_t)j] = std::max(lastr[(size_t)j], lastr[(size_t)j + 1]);
    for (int64_t j = j0; j < nsm;) {
      const int A = lastr[(size_t)j] / 32 + 1;
      const int q = pack ? (int)std::min<int64_t>(8 / A, nsm - j) : 1;
      h.cta_rb.push_back((int32_t)rb);
      h.cta_j.push_back((int32_t)(j | ((A - 1) << 16) | ((q - 1) << 20)));
      j += q;
    }
  }
  R.tbuf_total = to;
}

struct LayoutOff {
  size_t cut, poff, crb, cj, fwrb, fwl, twk, tws, tsj, tsb, tpart, toff, mc, xm1, state, part, tbuf, rscr;
};

}  // namespace

static int plan_build(const Params& prm, cudaStream_t stream, int64_t max_batch, int want_direct, Plan** out);

int plan_create_impl(int64_t N, int prec, double eps, int method, cudaStream_t stream, int64_t max_batch,
                     int want_direct, Plan** out) {
  Params prm;
  int st = derive_params(N, prec, eps, method, &prm);
  if (st != GBDLT_OK) return st;
  if (!(prm.method == GBDLT_METHOD_FAST && prm.grid != N)) return plan_build(prm, stream, max_batch, want_direct, out);
  // N not a power of two (grid.cu): the chain of a plan on the grid G > N, and
  // this plan's own arena for the N-point rule (and the direct layout)
  Params pi;
  st = derive_params(prm.grid, prec, eps, GBDLT_METHOD_FAST, &pi, prm.taylor_b);
  if (st != GBDLT_OK) return st;
  Plan* I = nullptr;
  st = plan_build(pi, stream, max_batch, 0, &I);
  if (st != GBDLT_OK) return st;
  Params po = prm;
  po.fast = false;
  Plan* O = nullptr;
  st = plan_build(po, stream, max_batch, want_direct, &O);
  if (st != GBDLT_OK) {
    free_plan(I);
    return st;
  }
  O->p = prm;
  O->inner = I;
  O->no_tma = I->no_tma;
  O->bcap = std::min(O->bcap, I->bcap);
  O->ws_bytes += I->ws_bytes;
  const size_t ts = prec == GBDLT_FP64 ? sizeof(double) : sizeof(float);
  const size_t rg = ts * (size_t)O->bcap * (size_t)prm.grid;
  if (dev_malloc(&O->rg_in, 2 * rg) != cudaSuccess) {
    cudaGetLastError();
    free_plan(O);
    return GBDLT_ERR_OOM;
  }
  O->rg_out = (char*)O->rg_in + rg;
  O->ws_bytes += 2 * rg;
  GridRules* R = nullptr;
  st = grid_rules_create(prm.grid, std::vector<Plan*>{O}, stream, &R);
  if (st == GBDLT_OK) {
    st = grid_attach(*I, R, nullptr, true);
    if (st != GBDLT_OK) grid_rules_free(R);
  }
  if (st != GBDLT_OK) {
    free_plan(O);
    return st;
  }
  O->ws_bytes += grid_rules_bytes(R) + ts * (size_t)I->bcap * (size_t)prm.grid;
  *out = O;
  return GBDLT_OK;
}

int plan_create_nodes(int64_t N, int prec, cudaStream_t stream, Plan** out) {
  Params q;
  int st = derive_params(N, prec, 0.0, GBDLT_METHOD_FAST, &q);
  if (st != GBDLT_OK) return st;
  q.fast = false;
  return plan_build(q, stream, 1, 0, out);
}

int plan_create_grid(int64_t G, int prec, double eps, double taylor_b, cudaStream_t stream, int64_t max_batch,
                     Plan** out) {
  if (G < 2 || (G & (G - 1))) return GBDLT_ERR_INVALID_ARG;
  Params q;
  int st = derive_params(G, prec, eps, GBDLT_METHOD_FAST, &q, taylor_b);
  if (st != GBDLT_OK) return st;
  return plan_build(q, stream, max_batch, 0, out);
}

static int plan_build(const Params& prm, cudaStream_t stream, int64_t max_batch, int want_direct, Plan** out) {
  const int64_t N = prm.N;
  const int prec = prm.prec;
  int st = GBDLT_OK;
  Plan* P = new (std::nothrow) Plan();
  if (!P) return GBDLT_ERR_OOM;
  P->p = prm;
  P->stream = stream;
  // staged FP32 FFT passes where they measured faster over a whole DLT + IDLT
  // (FP32 plans, 2^18 <= N <= 2^21; elsewhere neutral, or slower where their
  // persistent grid keeps the side stream's kernels off the SMs)
  P->no_tma = !(prm.prec == GBDLT_FP32 && N >= (1 << 18) && N <= (1 << 21));
  cudaGetDevice(&P->device);
  const size_t ts = prec == GBDLT_FP64 ? sizeof(double) : sizeof(float);
  const size_t cs = 2 * ts;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 1;
  }
  // recurrence layouts (host): the fast path's region on the cheb1 rows, and the
  // direct method's full rows at the Legendre nodes
  const int64_t batch_hint = max_batch > 0 ? max_batch : 1;
  LayoutHost hf, hd;
  if (prm.fast) {
    const int64_t H = N / 2;
    std::vector<int32_t> cut((size_t)std::max<int64_t>(H, 1), (int32_t)N);
    for (const Band& b : prm.bands)
      for (int64_t k = b.ka; k < b.kb; ++k) cut[(size_t)k] = (int32_t)b.ns;
    layout_build(P->rec, H, prm.seg, std::move(cut), (int)(prm.head / prm.seg), sms, batch_hint, true, hf);
  }
  P->has_direct = N > 1 && N <= kDirectMax && (prm.method == GBDLT_METHOD_DIRECT || want_direct);
  if (P->has_direct) {
    const int64_t H = (N + 1) / 2;
    // (512-column segments in either precision: a direct transform of N <= 512
    // is one segment, which the batch executor's fused direct launch relies on)
    layout_build(P->drec, H, 512, std::vector<int32_t>((size_t)H, (int32_t)N), 0, sms, batch_hint, false, hd);
  }
  RecLayout& R = P->rec;
  RecLayout& D = P->drec;
  const int npair = (prm.L + 1) / 2;
  // Taylor pairs in the plan's precision and in float-float, for either choice of
  // the l = 0 term (pairs of l = 0..L-1 or of l = 1..L-1)
  const int np1 = (prm.L + 1) / 2, np0 = prm.L / 2;
  const int p64max = std::max(taylor_p64(prm, 1, np1), taylor_p64(prm, 0, np0));
  const int pffmax = prec == GBDLT_FP64 ? std::max(np1 - taylor_p64(prm, 1, np1), np0 - taylor_p64(prm, 0, np0)) : 0;
  P->nfft_max = prm.fast ? std::max<int64_t>({(int64_t)prm.K * prm.M64, (int64_t)p64max, 1}) : 0;
  // FP32 band vectors of an FP64 plan (terms Mh..M-1); float-float vectors (band
  // terms M64..Mh-1, or the float-float Taylor pairs)
  const int64_t nfft32 = prm.fast && prec == GBDLT_FP64 ? (int64_t)prm.K * (prm.M - prm.Mh) : 0;
  const int64_t nfftff = prm.fast && prec == GBDLT_FP64
                             ? std::max<int64_t>((int64_t)prm.K * (prm.Mh - prm.M64), (int64_t)pffmax)
                             : 0;
  const bool scaled = nfft32 > 0 || nfftff > 0;
  // bands whose rows are few enough that their FFTs only touch two windows of
  // bins (four-step sizes only; see fft.cu, pruned passes)
  if (prm.fast && N > 4096) {
    int p2 = 0;
    while ((1ll << p2) < N) ++p2;
    const int64_t L1 = 1ll << (p2 / 2), L2 = N / L1;
    for (int s = 0; s < prm.K; ++s) {
      const int64_t Rs = prm.bands[s].kb / 2 + 2;
      if (2 * Rs > std::min(L1, L2)) break;
      P->prune_bands = s + 1;
      P->prune_R = (int)Rs;
    }
  }
  // FP32 plans with a head block above kHeadMM columns: the register-blocked
  // head kernels' tasks and per-item chunk partials (head.cu)
  const bool head_rb = prec == GBDLT_FP32 && prm.fast && prm.head > kHeadMM;
  std::vector<int4> rb_fwd, rb_trn;
  int64_t rb_part = 0;
  int rb_chunk = 0;
  if (head_rb) head_rb_tasks(prm.head, rb_fwd, rb_trn, &rb_part, &rb_chunk);
  {
    // batch capacity: as many vectors per pass as fit in ~512 MB of workspace
    const double per_item = 2.0 * P->nfft_max * N * cs + 2.0 * nfft32 * N * 8.0 + 2.0 * nfftff * N * 16.0 +
                            5.0 * N * ts +
                            16.0 * (R.nseg_total + D.nseg_total) +
                            8.0 * (R.tbuf_total + D.tbuf_total) + 8.0 * (double)rb_part +
                            8.0 * (double)R.tslots * R.S;
    P->bcap = std::max<int64_t>(1, std::min<int64_t>(4096, (int64_t)(512.0 * (1 << 20) / per_item)));
    if (max_batch > 0) P->bcap = std::min<int64_t>(P->bcap, max_batch);
  }
  const int64_t BC = P->bcap;
  // arena layout
  Arena A;
  size_t o_theta = A.take<double>(N), o_x = A.take<double>(N), o_w = A.take<double>(N),
         o_t = A.take<double>(N);
  size_t o_cn = A.take<double>(N + 1), o_ra = A.take<double>(N + 1024), o_rb = A.take<double>(N + 1024);
  size_t o_raff = A.take<float2>(N + 1024), o_rbff = A.take<float2>(N + 1024);
  size_t o_tw = A.take<double2>(4096);
  P->twN.B = N;
  P->tw4N.B = 4 * N;
  size_t o_twNlo = A.take<double2>(4096), o_twNhi = A.take<double2>(std::max<int64_t>(1, N / 4096));
  size_t o_tw4lo = A.take<double2>(4096), o_tw4hi = A.take<double2>(std::max<int64_t>(1, 4 * N / 4096));
  size_t o_twf = A.take<float2>(4096), o_twNflo = A.take<float2>(4096),
         o_twNfhi = A.take<float2>(std::max<int64_t>(1, N / 4096)), o_tw4flo = A.take<float2>(4096),
         o_tw4fhi = A.take<float2>(std::max<int64_t>(1, 4 * N / 4096));
  const bool fp64_tabs = prec == GBDLT_FP64 && prm.fast;
  size_t o_twfull = A.take<double2>(fp64_tabs && N > 4096 ? N : 1);
  size_t o_lf = A.take<double2>(4 * 4096);
  const bool stage_tabs = fp64_tabs && prm.K > 0 && prm.M > 0;
  size_t o_hnm = A.take<double>(stage_tabs ? (int64_t)prm.M64 * N : 1);
  size_t o_ar = A.take<RowAR>(stage_tabs ? N : 1);
  const int64_t nhead = prm.fast ? prm.head : 0;
  size_t o_lam = A.take<double>(std::max<int64_t>(nhead, 1)), o_lamf = A.take<float>(std::max<int64_t>(nhead, 1));
  // stored head products (FP64 plans): row k holds (nhead - k + 1) / 2 entries
  const bool head_tab = prec == GBDLT_FP64 && nhead > 0 && nhead <= kHeadTabMax;
  std::vector<int64_t> hoff;
  int64_t htab_n = 0;
  if (head_tab) {
    hoff.resize((size_t)nhead);
    for (int64_t k = 0; k < nhead; ++k) {
      hoff[(size_t)k] = htab_n;
      htab_n += (nhead - k + 1) / 2;
    }
  }
  size_t o_hoff = A.take<int64_t>(head_tab ? nhead : 1);
  size_t o_htab = A.take<double>(head_tab ? htab_n : 1);
  // the same products column by column (column n: rows k = n mod 2, ..., n), for
  // the transposed block: column n from offset hoffT[n]
  std::vector<int64_t> hoffT;
  int64_t htabT_n = 0;
  if (head_tab) {
    hoffT.resize((size_t)nhead);
    for (int64_t n = 0; n < nhead; ++n) {
      hoffT[(size_t)n] = htabT_n;
      htabT_n += n / 2 + 1;
    }
  }
  size_t o_hoffT = A.take<int64_t>(head_tab ? nhead : 1);
  size_t o_htabT = A.take<double>(head_tab ? htabT_n : 1);
  size_t o_lamp = A.take<float>(head_rb ? nhead + 2 * kHeadPad : 1);
  size_t o_rbt = A.take<int4>(head_rb ? (int64_t)(rb_fwd.size() + rb_trn.size()) : 1);
  size_t o_rbp = A.take<double>(head_rb ? BC * rb_part : 1);
  auto take_layout = [&](const RecLayout& L) {
    LayoutOff o;
    o.cut = A.take<int32_t>(L.H);
    o.poff = A.take<int64_t>(L.H);
    o.crb = A.take<int32_t>(L.ncta);
    o.cj = A.take<int32_t>(L.ncta);
    o.fwrb = A.take<int32_t>(L.nfw);
    o.fwl = A.take<int32_t>(32 * L.nfw);
    o.twk = A.take<int32_t>(32 * L.ntw);
    o.tws = A.take<int32_t>(32 * L.ntw);
    o.tsj = A.take<int32_t>(L.tslots);
    o.tsb = A.take<int32_t>(L.tsegs + 1);
    o.tpart = A.take<double>(BC * L.tslots * L.S);
    o.toff = A.take<int64_t>(L.nblocks);
    o.mc = A.take<int32_t>(L.nblocks);
    o.xm1 = A.take<double>(L.H);
    o.state = A.take<double2>(L.nseg_total);
    o.part = A.take<double2>(BC * L.nseg_total);
    o.tbuf = A.take<double>(BC * L.tbuf_total);
    o.rscr = A.take<double>(BC * ((L.nblocks + 63) / 64) * L.n_heavy);
    return o;
  };
  const LayoutOff of = take_layout(R), od = take_layout(D);
  auto bytes_block = [&](size_t b) {
    size_t o = A.off;
    A.off += (b + 255) & ~(size_t)255;
    return o;
  };
  size_t o_bufA = bytes_block((size_t)BC * P->nfft_max * (size_t)N * cs);
  size_t o_bufB = bytes_block((size_t)BC * P->nfft_max * (size_t)N * cs);
  size_t o_bufA32 = bytes_block((size_t)BC * nfft32 * (size_t)N * sizeof(float2));
  size_t o_bufAff = bytes_block((size_t)BC * nfftff * (size_t)N * sizeof(ffc));
  size_t o_bufBff = bytes_block((size_t)BC * nfftff * (size_t)N * sizeof(ffc));
  size_t o_tw4096ff = bytes_block(nfftff > 0 ? 4096 * sizeof(ffc) : 0);
  size_t o_twfullff = bytes_block(nfftff > 0 && N > 4096 ? (size_t)N * sizeof(ffc) : 0);
  size_t o_b32exp = A.take<int>(std::max<int64_t>(1, 2 * (int64_t)prm.K * prm.M));
  size_t o_h32 = A.take<float>(std::max<int64_t>(1, nfft32 > 0 ? (int64_t)(prm.M - prm.Mh) * N : 1));
  size_t o_hff = A.take<ffd>(std::max<int64_t>(1, nfftff > 0 ? (int64_t)(prm.Mh - prm.M64) * N : 1));
  size_t o_absmax = A.take<unsigned long long>(BC);
  size_t o_bufB32 = bytes_block((size_t)BC * nfft32 * (size_t)N * sizeof(float2));
  size_t o_v = bytes_block((size_t)BC * N * ts);
  size_t o_chat = bytes_block((size_t)BC * N * ts);
  size_t o_z = bytes_block((size_t)BC * N * ts);
  size_t o_tmp = bytes_block((size_t)BC * N * ts);
  size_t o_tmp2 = bytes_block((size_t)BC * N * ts);
  size_t o_status = A.take<int>(1);
  P->ws_bytes = A.off;
  if (dev_malloc(&P->arena, A.off) != cudaSuccess) {
    cudaGetLastError();
    free_plan(P);
    return GBDLT_ERR_OOM;
  }
  char* base = (char*)P->arena;
  P->theta = (double*)(base + o_theta);
  P->x = (double*)(base + o_x);
  P->w = (double*)(base + o_w);
  P->tN = (double*)(base + o_t);
  P->Cn = (double*)(base + o_cn);
  P->ra = (double*)(base + o_ra);
  P->rb = (double*)(base + o_rb);
  P->ra_ff = (float2*)(base + o_raff);
  P->rb_ff = (float2*)(base + o_rbff);
  P->tw4096 = (double2*)(base + o_tw);
  P->twN.lo = (double2*)(base + o_twNlo);
  P->twN.hi = (double2*)(base + o_twNhi);
  P->tw4N.lo = (double2*)(base + o_tw4lo);
  P->tw4N.hi = (double2*)(base + o_tw4hi);
  P->tw4096f = (float2*)(base + o_twf);
  P->twNf_lo = (float2*)(base + o_twNflo);
  P->twNf_hi = (float2*)(base + o_twNfhi);
  P->tw4Nf_lo = (float2*)(base + o_tw4flo);
  P->tw4Nf_hi = (float2*)(base + o_tw4fhi);
  P->twfull = fp64_tabs && N > 4096 ? (double2*)(base + o_twfull) : nullptr;
  P->lf_tab = fp64_tabs ? (double2*)(base + o_lf) : nullptr;
  P->Hnm = stage_tabs ? (double*)(base + o_hnm) : nullptr;
  P->row_ar = stage_tabs ? (RowAR*)(base + o_ar) : nullptr;
  P->head_lam = nhead > 0 ? (double*)(base + o_lam) : nullptr;
  P->head_lamf = nhead > 0 ? (float*)(base + o_lamf) : nullptr;
  P->head_off = head_tab ? (int64_t*)(base + o_hoff) : nullptr;
  P->head_tab = head_tab ? (double*)(base + o_htab) : nullptr;
  P->head_offT = head_tab ? (int64_t*)(base + o_hoffT) : nullptr;
  P->head_tabT = head_tab ? (double*)(base + o_htabT) : nullptr;
  if (head_rb) {
    P->head_lamp = (float*)(base + o_lamp);
    P->head_tasks = (int4*)(base + o_rbt);
    P->head_ntask_f = (int)rb_fwd.size();
    P->head_ntask_t = (int)rb_trn.size();
    P->head_part = (double*)(base + o_rbp);
    P->head_part_n = rb_part;
    P->head_rbc = rb_chunk;
  }
  auto place_layout = [&](RecLayout& L, const LayoutOff& o) {
    L.cut = (int32_t*)(base + o.cut);
    L.poff = (int64_t*)(base + o.poff);
    L.cta_rb = (int32_t*)(base + o.crb);
    L.cta_j = (int32_t*)(base + o.cj);
    L.fw_rb = (int32_t*)(base + o.fwrb);
    L.fw_lane = (int32_t*)(base + o.fwl);
    L.tw_k = (int32_t*)(base + o.twk);
    L.tw_slot = (int32_t*)(base + o.tws);
    L.tslot_j = (int32_t*)(base + o.tsj);
    L.tseg_begin = (int32_t*)(base + o.tsb);
    L.tpart = (double*)(base + o.tpart);
    L.toff = (int64_t*)(base + o.toff);
    L.bcutmax = (int32_t*)(base + o.mc);
    L.xm1 = (double*)(base + o.xm1);
    L.state = (double2*)(base + o.state);
    L.part = (double2*)(base + o.part);
    L.tbuf = (double*)(base + o.tbuf);
    L.rscratch = (double*)(base + o.rscr);
  };
  place_layout(R, of);
  place_layout(D, od);
  P->bufA = base + o_bufA;
  P->bufB = base + o_bufB;
  P->bufA32 = nfft32 > 0 ? base + o_bufA32 : nullptr;
  P->bufB32 = nfft32 > 0 ? base + o_bufB32 : nullptr;
  P->b32exp = scaled ? (int*)(base + o_b32exp) : nullptr;
  P->H32 = nfft32 > 0 ? (float*)(base + o_h32) : nullptr;
  P->Hff = nfftff > 0 ? (ffd*)(base + o_hff) : nullptr;
  P->bufAff = nfftff > 0 ? base + o_bufAff : nullptr;
  P->bufBff = nfftff > 0 ? base + o_bufBff : nullptr;
  P->tw4096_ff = nfftff > 0 ? (ffc*)(base + o_tw4096ff) : nullptr;
  P->twfull_ff = nfftff > 0 && N > 4096 ? (ffc*)(base + o_twfullff) : nullptr;
  P->absmax = scaled ? (unsigned long long*)(base + o_absmax) : nullptr;
  P->v = base + o_v;
  P->chat = base + o_chat;
  P->z = base + o_z;
  P->tmp = base + o_tmp;
  P->tmp2 = base + o_tmp2;
  P->status = (int*)(base + o_status);

  bool ok = true;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (bytes && cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
  };
  {
    std::vector<double> C = cn_table(N);
    up(P->Cn, C.data(), sizeof(double) * C.size());
    P->CN = C[(size_t)N];
    std::vector<double> ra((size_t)N + 1024), rb((size_t)N + 1024);
    for (int64_t n = 0; n < N + 1024; ++n) {
      ra[(size_t)n] = (double)(2 * n + 1) / (double)(n + 1);
      rb[(size_t)n] = (double)n / (double)(n + 1);
    }
    up(P->ra, ra.data(), sizeof(double) * ra.size());
    up(P->rb, rb.data(), sizeof(double) * rb.size());
    std::vector<float2> raf(ra.size()), rbf(rb.size());
    for (size_t i = 0; i < ra.size(); ++i) {
      const float ah = (float)ra[i], bh = (float)rb[i];
      raf[i] = make_float2(ah, (float)(ra[i] - (double)ah));
      rbf[i] = make_float2(bh, (float)(rb[i] - (double)bh));
    }
    up(P->ra_ff, raf.data(), sizeof(float2) * raf.size());
    up(P->rb_ff, rbf.data(), sizeof(float2) * rbf.size());
  }
  if (scaled) {
    // power-of-two scales of the FP32 and float-float band vectors: forward, the largest weight
    // C_n h_{m,n} (n >= ns, at n = ns) times 2^e <= 1; transposed, the largest
    // row factor (2 sin theta)^{-(m+1/2)} (at the band's first row) times 2^e <= 1
    const int K = prm.K, M = prm.M;
    std::vector<int> e((size_t)2 * K * M);
    for (int sb = 0; sb < K; ++sb) {
      const Band& bd = prm.bands[(size_t)sb];
      const double l2s = std::log2(2.0 * std::sin(((double)bd.ka + 0.5) * M_PI / (double)N));
      for (int m = 0; m < M; ++m) {
        const double l2w = (log_gM(m, (double)bd.ns) - std::log(2.0)) / std::log(2.0);
        e[(size_t)(sb * M + m)] = -(int)std::ceil(l2w);
        e[(size_t)(K * M + sb * M + m)] = (int)std::floor((m + 0.5) * l2s);
      }
    }
    up(P->b32exp, e.data(), sizeof(int) * e.size());
  }
  if (nhead > 0) {
    std::vector<double> lam = head_table(nhead);
    std::vector<float> lamf(lam.begin(), lam.end());
    up(P->head_lam, lam.data(), sizeof(double) * lam.size());
    up(P->head_lamf, lamf.data(), sizeof(float) * lamf.size());
    if (P->head_tab) up(P->head_off, hoff.data(), sizeof(int64_t) * hoff.size());
    if (P->head_tabT) up(P->head_offT, hoffT.data(), sizeof(int64_t) * hoffT.size());
    if (P->head_lamp) {
      // Lam' with kHeadPad zeros on each side: terms outside the triangle read zeros
      std::vector<float> lamp((size_t)(nhead + 2 * kHeadPad), 0.f);
      std::copy(lamf.begin(), lamf.end(), lamp.begin() + kHeadPad);
      up(P->head_lamp, lamp.data(), sizeof(float) * lamp.size());
      std::vector<int4> tasks(rb_fwd);
      tasks.insert(tasks.end(), rb_trn.begin(), rb_trn.end());
      up(P->head_tasks, tasks.data(), sizeof(int4) * tasks.size());
    }
  }
  auto upload_layout = [&](RecLayout& L, const LayoutHost& h) {
    if (L.H == 0) return;
    up(L.cut, h.cut.data(), sizeof(int32_t) * (size_t)L.H);
    up(L.poff, h.poff.data(), sizeof(int64_t) * (size_t)L.H);
    up(L.cta_rb, h.cta_rb.data(), sizeof(int32_t) * h.cta_rb.size());
    up(L.cta_j, h.cta_j.data(), sizeof(int32_t) * h.cta_j.size());
    up(L.fw_rb, h.fw_rb.data(), sizeof(int32_t) * h.fw_rb.size());
    up(L.fw_lane, h.fw_lane.data(), sizeof(int32_t) * h.fw_lane.size());
    up(L.tw_k, h.tw_k.data(), sizeof(int32_t) * h.tw_k.size());
    up(L.tw_slot, h.tw_slot.data(), sizeof(int32_t) * h.tw_slot.size());
    up(L.tslot_j, h.tslot_j.data(), sizeof(int32_t) * h.tslot_j.size());
    up(L.tseg_begin, h.tseg_begin.data(), sizeof(int32_t) * h.tseg_begin.size());
    up(L.toff, h.toff.data(), sizeof(int64_t) * h.toff.size());
    up(L.bcutmax, h.maxcut.data(), sizeof(int32_t) * h.maxcut.size());
  };
  upload_layout(R, hf);
  upload_layout(D, hd);
  if (cudaMemsetAsync(P->status, 0, sizeof(int), P->stream) != cudaSuccess) ok = false;
  if (!ok) {
    cudaGetLastError();
    free_plan(P);
    return GBDLT_ERR_CUDA;
  }
  st = launch_twiddle_init(*P);
  if (st == GBDLT_OK) st = launch_fft_tables_init(*P);
  if (st == GBDLT_OK) st = launch_stage_tables_init(*P);
  if (st == GBDLT_OK) st = launch_head_tab_init(*P);
  if (st == GBDLT_OK) st = launch_rec_xm1(*P, R, 0);
  if (st == GBDLT_OK) st = launch_rec_state_init(*P, R);
  if (st == GBDLT_OK) st = launch_legpts(*P, P->CN);
  // the direct layout's rows are the Legendre nodes just computed
  if (st == GBDLT_OK && P->has_direct) st = launch_rec_xm1(*P, D, 1);
  if (st == GBDLT_OK && P->has_direct) st = launch_rec_state_init(*P, D);
  if (st == GBDLT_OK && cudaStreamSynchronize(P->stream) != cudaSuccess) st = GBDLT_ERR_CUDA;
  if (st == GBDLT_OK) {
    int hs = 0;
    if (cudaMemcpy(&hs, P->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = GBDLT_ERR_CUDA;
    else if (hs & 1)
      st = GBDLT_ERR_NOT_CONVERGED;
  }
  if (st != GBDLT_OK) {
    cudaGetLastError();
    free_plan(P);
    return st;
  }
  *out = P;
  return GBDLT_OK;
}

// ---------------------------------------------------------------------------
// transform chains
// ---------------------------------------------------------------------------
namespace {

// the FFT buffer that does not hold `p`
inline void* other(Plan& P, const void* p) { return p == P.bufA ? P.bufB : P.bufA; }

// A branch of a chain on the plan's side stream.  GB300 retires 2 FP64 operations
// per SM and clock against 128 FP32 ones, and the FP64 kernels issue an
// instruction in about one cycle of ten; the float-float and FP32 transforms of a
// stage (independent of its FP64 transforms and recurrence, disjoint buffers)
// therefore run on the side stream beside the FP64 work, and the stage's
// epilogue waits for both.  Not while profiling (the per-kernel events assume one
// stream).  Inside a capture the side stream joins the caller's graph as a branch.
struct Side {
  Plan& P;
  cudaStream_t main;
  bool on = false;
  Side(Plan& p, bool want) : P(p), main(p.stream) {
    if (!want || (P.prof && P.prof->on)) return;
    if (!P.side && !P.side_broken) {
      if (cudaStreamCreateWithFlags(&P.side, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&P.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&P.ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        P.side_broken = true;
      }
    }
    if (P.side_broken || !P.side) return;
    if (cudaEventRecord(P.ev_fork, main) != cudaSuccess || cudaStreamWaitEvent(P.side, P.ev_fork, 0) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    on = true;
  }
  // launches between enter() and leave() go to the side stream
  void enter() {
    if (on) P.stream = P.side;
  }
  void leave() { P.stream = main; }
  // the plan stream waits for the side branch
  int join() {
    P.stream = main;
    if (!on) return GBDLT_OK;
    on = false;
    if (cudaEventRecord(P.ev_join, P.side) != cudaSuccess || cudaStreamWaitEvent(main, P.ev_join, 0) != cudaSuccess)
      return GBDLT_ERR_CUDA;
    return GBDLT_OK;
  }
  ~Side() { join(); }
};

// The band FFTs: terms m < M64 in precision T from `a` (result returned); in
// FP64 plans terms M64 <= m < Mh in float-float from the plan's float-float band
// buffers (result in *yff) and terms m >= Mh in FP32 from its FP32 ones (*y32).
// The float-float and FP32 ones go to the side branch `sd` (joined by the caller).
inline bool side_bands(const Plan& P) {
  return P.p.K > 0 && ((P.p.Mh > P.p.M64 && P.bufAff) || (P.p.M > P.p.Mh && P.bufA32));
}
template <typename T>
const C2<T>* band_ffts(Plan& P, Side& sd, void* a, int64_t nb, int dir, int transposed, const ffc** yff,
                       const float2** y32) {
  const int Ml = P.p.M - P.p.Mh, Mf = P.p.Mh - P.p.M64;
  *y32 = nullptr;
  *yff = nullptr;
  const C2<T>* y = nullptr;
  if (P.p.K > 0 && P.p.M64 > 0)
    y = (const C2<T>*)launch_fft_bands<T>(P, a, other(P, a), nb, dir, transposed, P.p.M64);
  sd.enter();
  if (P.p.K > 0 && Mf > 0 && P.bufAff)
    *yff = (const ffc*)launch_fft_bands<ffd>(P, P.bufAff, P.bufBff, nb, dir, transposed, Mf);
  if (P.p.K > 0 && Ml > 0 && P.bufA32)
    *y32 = (const float2*)launch_fft_bands<float>(P, P.bufA32, P.bufB32, nb, dir, transposed, Ml);
  sd.leave();
  return y;
}

// chat = M c (Sec. 3); also leaves v (values on the cheb1 grid) in P.v
// In FP32 plans the dense head block (FP32-pipe work that reads only c) runs on the
// side stream beside the rest of leg2cheb and writes its columns to P.z as
// doubles; the A4 epilogue adds them.  (FP64 plans add it in place at the end: it
// is FP64 work like the rest of the chain.)
template <typename T>
int run_leg2cheb(Plan& P, const T* c, T* chat, int64_t nb) {
  const int64_t KM = (int64_t)P.p.K * P.p.M;
  T* vrec = (T*)P.tmp;
  T* v = (T*)P.v;
  int st = GBDLT_OK;
  const bool head_side = is_f32<T> && P.p.head > 0;
  double* hb = head_side ? (double*)P.z : nullptr;
  Side hs(P, head_side);
  if (head_side) {
    hs.enter();
    st = launch_head_fwd<T>(P, c, chat, nb, hb);
    hs.leave();
    if (st) return st;
  }
  const C2<T>* Y = nullptr;
  const ffc* Yff = nullptr;
  const float2* Y32 = nullptr;
  {
    if (KM > 0) {
      st = launch_absmax<T>(P, c, nb);
      if (st) return st;
      st = launch_l2c_pro<T>(P, c, (C2<T>*)P.bufA, (ffc*)P.bufAff, (float2*)P.bufA32, nb);
      if (st) return st;
    }
    // band FFTs (FP32-pipe ones on the side branch) beside the recurrence region
    Side sd(P, KM > 0 && side_bands(P));
    if (KM > 0) Y = band_ffts<T>(P, sd, P.bufA, nb, +1, 0, &Yff, &Y32);
    st = launch_rec_forward<T>(P, P.rec, c, vrec, nb);
    const int sj = sd.join();
    if (st) return st;
    if (sj) return sj;
  }
  st = launch_l2c_epi<T>(P, Y, Yff, Y32, vrec, v, nb);
  if (st) return st;
  st = launch_a4_pro<T>(P, v, (C2<T>*)P.bufA, nb);
  if (st) return st;
  const C2<T>* F = (const C2<T>*)launch_fft<T>(P, P.bufA, P.bufB, nb, -1);
  st = hs.join();
  if (st) return st;
  st = launch_a4_epi<T>(P, F, chat, nb, hb);
  if (st) return st;
  // columns below the head: P.v lacks them, so chains that go on to the Taylor
  // NDCT take its l = 0 term from chat (run_dlt_tail)
  return head_side ? GBDLT_OK : launch_head_fwd<T>(P, c, chat, nb);
}

// The FP64 and float-float FFTs of a Taylor stage (inputs in bufA / bufAff):
// one mixed pair of launches when both kinds have vectors at a four-step size
// (FP64 plans, by the fft_mix mode and N), else the float-float ones on the side stream beside
// the FP64 ones.  Results: *y (the FP64 buffer the passes end in), *yff.
template <typename T>
int taylor_ffts(Plan& P, int64_t n64, int64_t nff, int dir, const void** y, const ffc** yff) {
  *yff = nullptr;
  if constexpr (is_f64<T>) {
    const bool mix = P.fft_mix == 2 || (P.fft_mix == 1 && P.p.N >= kFftMixMinN);
    if (mix && nff > 0 && n64 > 0 && P.p.N > 4096) {
      launch_fft_mix(P, P.bufA, P.bufB, n64, P.bufAff, P.bufBff, nff, dir);
      *y = P.bufB;
      *yff = (const ffc*)P.bufBff;
      return check_launch();
    }
  }
  Side sd(P, nff > 0);
  *y = launch_fft<T>(P, P.bufA, P.bufB, n64, dir);
  sd.enter();
  if (nff > 0) *yff = (const ffc*)launch_fft<ffd>(P, P.bufAff, P.bufBff, nff, dir);
  return sd.join();
}

// forward declaration (defined below)
template <typename T>
int run_taylor(Plan& P, const T* chat, const T* v, T* f, int inc0, int64_t nb);

// f = Taylor NDCT of P.chat after run_leg2cheb: the l = 0 term is v itself
// (values on the cheb1 grid) when the plan has no head block, else it is one
// more transformed term of chat (for even L the pair count is the same)
template <typename T>
int run_dlt_tail(Plan& P, T* out, int64_t nb) {
  if (P.p.head > 0) return run_taylor<T>(P, (const T*)P.chat, nullptr, out, 1, nb);
  return run_taylor<T>(P, (const T*)P.chat, (const T*)P.v, out, 0, nb);
}

// Taylor NDCT (Sec. 2): f = [v] + sum_{l} ...; inc0 = 1 includes l = 0 (standalone chebeval)
template <typename T>
int run_taylor(Plan& P, const T* chat, const T* v, T* f, int inc0, int64_t nb) {
  const int npair = inc0 ? (P.p.L + 1) / 2 : P.p.L / 2;
  if (npair == 0) {
    if (!inc0) return cudaMemcpyAsync(f, v, sizeof(T) * P.p.N * nb, cudaMemcpyDeviceToDevice,
                                      P.stream) == cudaSuccess
                          ? GBDLT_OK
                          : GBDLT_ERR_CUDA;
  }
  // pairs of small terms in float-float (FP64 plans), scaled by the input's exponent
  ffc* Uff = (ffc*)P.bufAff;
  const int P64 = Uff ? taylor_p64(P.p, inc0, npair) : npair;
  if (P64 == npair) Uff = nullptr;
  int st = Uff ? launch_absmax<T>(P, chat, nb) : GBDLT_OK;
  if (st) return st;
  st = launch_tay_pro<T>(P, chat, (C2<T>*)P.bufA, Uff, inc0, npair, nb);
  if (st) return st;
  const C2<T>* Y = nullptr;
  const ffc* Yff = nullptr;
  {
    const void* y = nullptr;
    st = taylor_ffts<T>(P, nb * P64, Uff ? nb * (npair - P64) : 0, +1, &y, &Yff);
    if (st) return st;
    Y = (const C2<T>*)y;
  }
  return launch_tay_epi<T>(P, Y, Yff, v, f, inc0, npair, nb);
}

// transposed chain: out = [D_s] P^T [D_w] g (idlt when weighted), Sec. 4.
// Without a head block the l = 0 Taylor term enters in value space (z = g + ...);
// with one, every term goes through the coefficient-space sum u = T^T-type
// transposed Taylor sum, whose first `head` entries feed the transposed head block.
template <typename T>
int run_transposed(Plan& P, const T* g, T* out, int use_w, int scale_s, int64_t nb) {
  const int64_t KM = (int64_t)P.p.K * P.p.M;
  const int64_t head = P.p.head;
  const int inc0 = head > 0 ? 1 : 0;
  const int npair = inc0 ? (P.p.L + 1) / 2 : P.p.L / 2;  // l = 0..L-1, or 1..L-1
  T* z = (T*)P.z;
  T* rect = (T*)P.tmp;
  T* uhead = (T*)P.chat;  // first `head` coefficients of u (batch stride N)
  ffc* Uff = (ffc*)P.bufAff;
  const int P64 = Uff ? taylor_p64(P.p, inc0, npair) : npair;
  if (P64 == npair) Uff = nullptr;
  int st = (KM > 0 || Uff) ? launch_absmax<T>(P, g, nb) : GBDLT_OK;
  if (st) return st;
  const C2<T>* Y = nullptr;  // A4^T FFT output
  if (npair > 0) {
    st = launch_tayt_pro<T>(P, g, use_w, (C2<T>*)P.bufA, Uff, inc0, npair, nb);
    if (st) return st;
    const void* F = nullptr;
    const ffc* Fff = nullptr;
    st = taylor_ffts<T>(P, nb * P64, Uff ? nb * (npair - P64) : 0, -1, &F, &Fff);
    if (st) return st;
    void* q = other(P, F);
    st = launch_tayt_epi<T>(P, (const C2<T>*)F, Fff, (C2<T>*)q, head > 0 ? uhead : nullptr, inc0, npair, nb,
                            head);
    if (st) return st;
    Y = (const C2<T>*)launch_fft<T>(P, q, other(P, q), nb, +1);
  }
  // The transposed head block (reads u[0:head]) on the side stream beside the rest
  // of the chain, its scaled columns into P.tmp2 as doubles; the transposed
  // leg2cheb epilogue adds them.  FP32 plans: FP32-pipe work.  FP64 plans with the
  // stored products: a latency-bound kernel (about 70 % of the FP64 pipe) that
  // fills gaps of the FP64 work beside it.
  const bool head_side = (is_f32<T> || P.head_tab) && head > 0 && npair > 0;
  double* hb = head_side ? (double*)P.tmp2 : nullptr;
  Side hsd(P, head_side);
  if (head_side) {
    hsd.enter();
    st = launch_head_t<T>(P, uhead, out, scale_s, nb, hb);
    hsd.leave();
    if (st) return st;
  }
  void* U = Y ? other(P, Y) : P.bufA;
  // the l = 0 term in value space: the rows themselves, or (rows of an outer
  // rule, grid.cu) the rows summed onto their grid points
  const T* g0 = g;
  int w0 = use_w;
  if (!inc0 && P.rg_rules) {
    st = launch_grid_scatter<T>(P, g, use_w, (T*)P.rg_g, nb);
    if (st) return st;
    g0 = (const T*)P.rg_g;
    w0 = 0;
  }
  st = launch_l2ct_pro<T>(P, Y, inc0 ? nullptr : g0, inc0 ? 0 : w0, z, (C2<T>*)U, (ffc*)P.bufAff,
                          (float2*)P.bufA32, nb);
  if (st) return st;
  const C2<T>* F2 = nullptr;
  const ffc* Fff = nullptr;
  const float2* F32 = nullptr;
  {
    Side sd(P, KM > 0 && side_bands(P));
    if (KM > 0) F2 = band_ffts<T>(P, sd, U, nb, -1, 1, &Fff, &F32);
    st = launch_rec_transpose<T>(P, P.rec, z, rect, nb);
    const int sj = sd.join();
    if (st) return st;
    if (sj) return sj;
  }
  st = hsd.join();
  if (st) return st;
  st = launch_l2ct_epi<T>(P, F2, Fff, F32, rect, out, scale_s, nb, hb);
  if (st) return st;
  return head_side ? GBDLT_OK : launch_head_t<T>(P, uhead, out, scale_s, nb);
}

// out = M^T y: z = A4^T y, then P_cheb^T z
template <typename T>
int run_leg2cheb_t(Plan& P, const T* y, T* out, int64_t nb) {
  const int64_t KM = (int64_t)P.p.K * P.p.M;
  T* z = (T*)P.z;
  T* rect = (T*)P.tmp;
  int st = KM > 0 ? launch_absmax<T>(P, y, nb) : GBDLT_OK;
  if (st) return st;
  st = launch_fcs_pro<T>(P, y, (C2<T>*)P.bufA, 1, nb);
  if (st) return st;
  const void* Y = launch_fft<T>(P, P.bufA, P.bufB, nb, +1);
  void* U = other(P, Y);
  st = launch_l2ct_pro<T>(P, (const C2<T>*)Y, nullptr, 0, z, (C2<T>*)U, (ffc*)P.bufAff, (float2*)P.bufA32, nb);
  if (st) return st;
  const C2<T>* F2 = nullptr;
  const ffc* Fff = nullptr;
  const float2* F32 = nullptr;
  {
    Side sd(P, KM > 0 && side_bands(P));
    if (KM > 0) F2 = band_ffts<T>(P, sd, U, nb, -1, 1, &Fff, &F32);
    st = launch_rec_transpose<T>(P, P.rec, z, rect, nb);
    const int sj = sd.join();
    if (st) return st;
    if (sj) return sj;
  }
  st = launch_l2ct_epi<T>(P, F2, Fff, F32, rect, out, 0, nb);
  if (st) return st;
  return launch_head_t<T>(P, y, out, 0, nb);
}

template <typename T>
int run_chebeval_t(Plan& P, const T* g, T* out, int64_t nb) {
  const int npair = (P.p.L + 1) / 2;  // l = 0..L-1
  ffc* Uff = (ffc*)P.bufAff;
  const int P64 = Uff ? taylor_p64(P.p, 1, npair) : npair;
  if (P64 == npair) Uff = nullptr;
  int st = Uff ? launch_absmax<T>(P, g, nb) : GBDLT_OK;
  if (st) return st;
  st = launch_tayt_pro<T>(P, g, 0, (C2<T>*)P.bufA, Uff, 1, npair, nb);
  if (st) return st;
  const void* F = nullptr;
  const ffc* Fff = nullptr;
  st = taylor_ffts<T>(P, nb * P64, Uff ? nb * (npair - P64) : 0, -1, &F, &Fff);
  if (st) return st;
  return launch_tayt_epi<T>(P, (const C2<T>*)F, Fff, nullptr, out, 1, npair, nb);
}


// Direct method: the sums of Eq. (1) and (2) by the recurrence at the Legendre
// nodes over all columns (rows k and N-1-k share one recurrence).
//   DLT     f = P c
//   DLT^T   out = P^T g
//   IDLT    c = D_s P^T D_w f  (weights on the rows, n + 1/2 on the reduction)
//   IDLT^T  out = D_w P D_s g
template <typename T>
int run_direct(Plan& P, int op, const T* in, T* out, int64_t nb) {
  RecLayout& D = P.drec;
  switch (op) {
    case OP_DLT:
      return launch_rec_forward<T>(P, D, in, out, nb);
    case OP_DLT_T:
      return launch_rec_transpose<T>(P, D, in, out, nb, nullptr, 0);
    case OP_IDLT:
      return launch_rec_transpose<T>(P, D, in, out, nb, P.w, 1);
    case OP_IDLT_T: {
      T* sg = (T*)P.tmp2;
      int st = launch_scale<T>(P, in, sg, 1, nb);
      if (st) return st;
      st = launch_rec_forward<T>(P, D, sg, out, nb);
      if (st) return st;
      return launch_scale<T>(P, out, out, 2, nb);
    }
  }
  return GBDLT_ERR_INVALID_ARG;
}

// A plan whose N is not a power of two (grid.cu): pad the inputs to the inner
// plan's grid G, run its chain (rows: this plan's N-point rule), keep the first
// N outputs of each item.
template <typename T>
int run_grid(Plan& O, int op, const T* in, T* out, int64_t nb) {
  Plan& I = *O.inner;
  I.stream = O.stream;
  I.prof = O.prof;
  const int64_t N = O.p.N, G = I.p.N;
  T* xi = (T*)O.rg_in;
  T* xo = (T*)O.rg_out;
  int st = launch_grid_pad<T>(O, in, xi, N, G, nb);
  if (st == GBDLT_OK) {
    switch (op) {
      case OP_L2C:
        st = run_leg2cheb<T>(I, xi, xo, nb);
        break;
      case OP_L2C_T:
        st = run_leg2cheb_t<T>(I, xi, xo, nb);
        break;
      case OP_CHEB:
        st = run_taylor<T>(I, xi, nullptr, xo, 1, nb);
        break;
      case OP_CHEB_T:
        st = run_chebeval_t<T>(I, xi, xo, nb);
        break;
      case OP_DLT:
        st = run_leg2cheb<T>(I, xi, (T*)I.chat, nb);
        if (st == GBDLT_OK) st = run_dlt_tail<T>(I, xo, nb);
        break;
      case OP_DLT_T:
        st = run_transposed<T>(I, xi, xo, 0, 0, nb);
        break;
      case OP_IDLT:
        st = run_transposed<T>(I, xi, xo, 1, 1, nb);
        break;
      case OP_IDLT_T: {
        // out = D_w P D_s g: D_s on the padded vector, D_w (this rule's weights) at the end
        T* sg = (T*)I.tmp2;
        st = launch_scale<T>(I, xi, sg, 1, nb);
        if (st == GBDLT_OK) st = run_leg2cheb<T>(I, sg, (T*)I.chat, nb);
        if (st == GBDLT_OK) st = run_dlt_tail<T>(I, xo, nb);
        break;
      }
      default:
        st = GBDLT_ERR_INVALID_ARG;
    }
  }
  if (st == GBDLT_OK) st = launch_grid_cut<T>(O, xo, out, N, G, nb);
  if (st == GBDLT_OK && op == OP_IDLT_T) st = launch_scale<T>(O, out, out, 2, nb);
  I.prof = nullptr;
  return st;
}

template <typename T>
int run_one(Plan& P, int op, int method, const T* in, T* out, int64_t nb) {
  const int64_t N = P.p.N;
  if (N == 1) {
    // every operator is the identity at N = 1 (P_0 = T_0 = 1, w_0 = 2, s_0 = 1/2)
    return cudaMemcpyAsync(out, in, sizeof(T) * nb, cudaMemcpyDeviceToDevice, P.stream) == cudaSuccess
               ? GBDLT_OK
               : GBDLT_ERR_CUDA;
  }
  const bool transform = op == OP_DLT || op == OP_DLT_T || op == OP_IDLT || op == OP_IDLT_T;
  if (transform && method == GBDLT_METHOD_DIRECT) {
    if (!P.has_direct) return GBDLT_ERR_UNSUPPORTED_N;
    return run_direct<T>(P, op, in, out, nb);
  }
  if (P.inner) return run_grid<T>(P, op, in, out, nb);
  if (!P.p.fast) return GBDLT_ERR_UNSUPPORTED_N;  // a direct-method plan for N that is not a power of two
  switch (op) {
    case OP_L2C:
      return run_leg2cheb<T>(P, in, out, nb);
    case OP_L2C_T:
      return run_leg2cheb_t<T>(P, in, out, nb);
    case OP_CHEB:
      return run_taylor<T>(P, in, nullptr, out, 1, nb);
    case OP_CHEB_T:
      return run_chebeval_t<T>(P, in, out, nb);
    case OP_DLT: {
      int st = run_leg2cheb<T>(P, in, (T*)P.chat, nb);
      if (st) return st;
      return run_dlt_tail<T>(P, out, nb);
    }
    case OP_DLT_T:
      return run_transposed<T>(P, in, out, 0, 0, nb);
    case OP_IDLT:
      return run_transposed<T>(P, in, out, 1, 1, nb);
    case OP_IDLT_T: {
      // out = D_w P D_s g (a plan carrying other rules has no weights of its own
      // to apply: run_grid applies the rule's)
      if (P.rg_rules) return GBDLT_ERR_INVALID_ARG;
      T* sg = (T*)P.tmp2;
      int st = launch_scale<T>(P, in, sg, 1, nb);
      if (st) return st;
      st = run_leg2cheb<T>(P, sg, (T*)P.chat, nb);
      if (st) return st;
      st = run_dlt_tail<T>(P, out, nb);
      if (st) return st;
      return launch_scale<T>(P, out, out, 2, nb);
    }
  }
  return GBDLT_ERR_INVALID_ARG;
}

}  // namespace

int run_op(gbdlt_plan plan, int op, const void* in, void* out, int64_t batch) {
  if (!plan) return GBDLT_ERR_INVALID_ARG;
  return run_op_method(plan, op, reinterpret_cast<Plan*>(plan)->p.method, in, out, batch);
}

static int run_chain(Plan& P, int op, int method, const void* in, void* out, int64_t batch);

int run_op_method(gbdlt_plan plan, int op, int method, const void* in, void* out, int64_t batch) {
  if (!plan || batch < 0) return GBDLT_ERR_INVALID_ARG;
  if (method != GBDLT_METHOD_FAST && method != GBDLT_METHOD_DIRECT) return GBDLT_ERR_INVALID_ARG;
  if (batch == 0) return GBDLT_OK;  // nothing to do; the pointers are not read
  if (!in || !out) return GBDLT_ERR_INVALID_ARG;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  const size_t es = P.p.prec == GBDLT_FP64 ? 8 : 4;
  if (((uintptr_t)in % es) || ((uintptr_t)out % es)) return GBDLT_ERR_INVALID_ARG;
  {
    const char* a = (const char*)in;
    const char* ae = a + (size_t)batch * P.p.N * es;
    const char* b = (const char*)out;
    const char* be = b + (size_t)batch * P.p.N * es;
    if (a < be && b < ae) return GBDLT_ERR_INVALID_ARG;  // overlap
  }
  // direct execution: profiling, a capturing caller stream, or a broken cache
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(P.stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;  // cannot tell: do not capture
  }
  if ((P.prof && P.prof->on) || cs != cudaStreamCaptureStatusNone || (P.graphs && P.graphs->broken))
    return run_chain(P, op, method, in, out, batch);
  if (!P.graphs) {
    GraphCache* G = new (std::nothrow) GraphCache();
    if (!G) return run_chain(P, op, method, in, out, batch);
    P.graphs = G;
    if (cudaStreamCreateWithFlags(&G->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&G->out, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      G->broken = true;
      return run_chain(P, op, method, in, out, batch);
    }
  }
  GraphCache& G = *P.graphs;
  ++G.tick;
  const bool with_nodes = P.nodes_pending && op != OP_L2C && op != OP_L2C_T;
  GraphEntry* E = nullptr;
  for (GraphEntry& x : G.e)
    if (x.op == op && x.method == method && x.in == in && x.out == out && x.batch == batch && x.nodes == with_nodes)
      E = &x;
  if (!E) {
    if (G.e.size() >= kGraphCacheSize) {
      size_t lru = 0;
      for (size_t i = 1; i < G.e.size(); ++i)
        if (G.e[i].last < G.e[lru].last) lru = i;
      if (G.e[lru].exec) cudaGraphExecDestroy(G.e[lru].exec);
      G.e.erase(G.e.begin() + (long)lru);
    }
    GraphEntry x;
    x.op = op;
    x.method = method;
    x.nodes = with_nodes;
    x.in = in;
    x.out = out;
    x.batch = batch;
    G.e.push_back(x);
    E = &G.e.back();
  }
  E->last = G.tick;
  if (++E->calls < 2) return run_chain(P, op, method, in, out, batch);
  // fork onto the internal stream
  if (cudaEventRecord(G.in, P.stream) != cudaSuccess || cudaStreamWaitEvent(G.s, G.in, 0) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  if (!E->exec) {
    cudaStream_t user = P.stream;
    P.stream = G.s;
    int st = GBDLT_OK;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(G.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = GBDLT_ERR_CUDA;
    } else {
      // kernels recorded into the graph are counted when the graph is launched
      const uint64_t c0 = launches_now();
      st = run_chain(P, op, method, in, out, batch);
      uncount_launches(launches_now() - c0);
      if (cudaStreamEndCapture(G.s, &graph) != cudaSuccess) st = st ? st : GBDLT_ERR_CUDA;
    }
    P.stream = user;
    if (st == GBDLT_OK && graph && cudaGraphInstantiate(&E->exec, graph, 0) == cudaSuccess) {
      size_t n = 0;
      if (cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess) {
        std::vector<cudaGraphNode_t> nodes(n);
        if (n && cudaGraphGetNodes(graph, nodes.data(), &n) == cudaSuccess)
          for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++E->kernels;
          }
      }
    } else {
      E->exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    if (!E->exec) {
      // capture did not work: the work was not done; run it directly from now on
      cudaGetLastError();
      G.broken = true;
      if (cudaEventRecord(G.out, G.s) == cudaSuccess) cudaStreamWaitEvent(P.stream, G.out, 0);
      return st ? st : run_chain(P, op, method, in, out, batch);
    }
  }
  if (cudaGraphLaunch(E->exec, G.s) != cudaSuccess) return GBDLT_ERR_CUDA;
  count_launch((int)E->kernels);
  if (with_nodes) P.nodes_pending = false;  // the replayed chain ran the node kernel
  if (cudaEventRecord(G.out, G.s) != cudaSuccess || cudaStreamWaitEvent(P.stream, G.out, 0) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  return GBDLT_OK;
}

// A deferred node refresh (gbdlt_legpts without outputs) starts with the next
// chain that reads the nodes: as a branch on the plan's node stream beside the
// chain's first stages when the chain is the FFT-based one of a power-of-two
// plan (the node kernel is FP64-pipe work, the stages before the Taylor step do
// not read the nodes), else in the plan stream before the chain.  Not as a
// branch while profiling (the per-kernel events assume one stream).
static int nodes_start(Plan& P, bool branch) {
  if (!P.nodes_pending) return GBDLT_OK;
  P.nodes_pending = false;
  if (branch && !(P.prof && P.prof->on)) {
    if (!P.node_s && (cudaStreamCreateWithFlags(&P.node_s, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreateWithFlags(&P.node_fork, cudaEventDisableTiming) != cudaSuccess ||
                      cudaEventCreateWithFlags(&P.node_join, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      return GBDLT_ERR_CUDA;
    }
    if (cudaEventRecord(P.node_fork, P.stream) != cudaSuccess ||
        cudaStreamWaitEvent(P.node_s, P.node_fork, 0) != cudaSuccess)
      return GBDLT_ERR_CUDA;
    cudaStream_t main = P.stream;
    P.stream = P.node_s;
    // two blocks (8 warps) per SM keep the FP64 pipe busy and leave the rest of
    // each SM to the chain's kernels
    int st = launch_legpts(P, P.CN, 2);
    P.stream = main;
    if (st) return st;
    if (cudaEventRecord(P.node_join, P.node_s) != cudaSuccess) return GBDLT_ERR_CUDA;
    P.node_branch_open = true;
    return GBDLT_OK;
  }
  return launch_legpts(P, P.CN);
}

int nodes_ready(Plan& P) {
  if (!P.node_branch_open) return GBDLT_OK;
  P.node_branch_open = false;
  return cudaStreamWaitEvent(P.stream, P.node_join, 0) == cudaSuccess ? GBDLT_OK : GBDLT_ERR_CUDA;
}

static int run_chain(Plan& P, int op, int method, const void* in, void* out, int64_t batch) {
  const int64_t N = P.p.N;
  if (P.nodes_pending && op != OP_L2C && op != OP_L2C_T) {
    const bool branch = method == GBDLT_METHOD_FAST && P.p.fast && !P.inner && P.p.N > 1;
    int st = nodes_start(P, branch);
    if (st) return st;
  }
  for (int64_t i = 0; i < batch; i += P.bcap) {
    const int64_t nb = std::min<int64_t>(P.bcap, batch - i);
    P.rg_item0 = i;  // the rule table of a grid plan's batch items (grid.cu)
    int st;
    if (P.p.prec == GBDLT_FP64)
      st = run_one<double>(P, op, method, (const double*)in + i * N, (double*)out + i * N, nb);
    else
      st = run_one<float>(P, op, method, (const float*)in + i * N, (float*)out + i * N, nb);
    if (st) {
      nodes_ready(P);
      return st;
    }
  }
  // every branch rejoins the plan stream (a capture needs it; a chain whose
  // readers all ran has joined already)
  if (int st = nodes_ready(P)) return st;
  return check_launch();
}


}  // namespace gbdlt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace gbdlt;

struct gbdlt_plan_s {};  // opaque tag; the pointer is a gbdlt::Plan

extern "C" {

static void fill_public(const Params& q, size_t ws, gbdlt_params* out) {
  std::memset(out, 0, sizeof(*out));
  out->N = q.N;
  out->prec = q.prec;
  out->eps = q.eps;
  out->L = q.L;
  out->M = q.M;
  out->K = q.K;
  for (int s = 0; s < q.K && s < GBDLT_MAX_BANDS; ++s) {
    out->band_ns[s] = q.bands[s].ns;
    out->band_ka[s] = q.bands[s].ka;
    out->band_kb[s] = q.bands[s].kb;
  }
  out->rec_steps = q.rec_steps;
  out->seg_len = q.seg;
  out->flops_dlt = q.flops_dlt;
  out->bytes_dlt = q.bytes_dlt;
  out->bytes_idlt = q.bytes_idlt;
  out->workspace_bytes = ws;
  out->method = q.method;
  out->direct_steps = q.direct_steps;
  out->head = q.head;
  out->M_fp32 = q.M - q.Mh;
  out->M_ff = q.Mh - q.M64;
  out->L_ff = q.L - q.Lff;
  out->grid_n = q.grid;
}

int gbdlt_plan_params_ex(int64_t N, int prec, double eps, int method, gbdlt_params* out) {
  if (!out) return GBDLT_ERR_INVALID_ARG;
  Params q;
  int st = derive_params(N, prec, eps, method, &q);
  if (st) return st;
  fill_public(q, 0, out);
  return GBDLT_OK;
}

int gbdlt_plan_params(int64_t N, int prec, double eps, gbdlt_params* out) {
  return gbdlt_plan_params_ex(N, prec, eps, GBDLT_METHOD_AUTO, out);
}

int gbdlt_plan_create_ex(int64_t N, int prec, double eps, int method, void* cuda_stream, gbdlt_plan* out) {
  if (!out) return GBDLT_ERR_INVALID_ARG;
  *out = nullptr;
  Plan* P = nullptr;
  int st = plan_create_impl(N, prec, eps, method, (cudaStream_t)cuda_stream, 0, 0, &P);
  if (st) return st;
  *out = reinterpret_cast<gbdlt_plan>(P);
  return GBDLT_OK;
}

int gbdlt_plan_create(int64_t N, int prec, double eps, void* cuda_stream, gbdlt_plan* out) {
  return gbdlt_plan_create_ex(N, prec, eps, GBDLT_METHOD_AUTO, cuda_stream, out);
}

int gbdlt_plan_destroy(gbdlt_plan plan) {
  if (!plan) return GBDLT_ERR_INVALID_ARG;
  Plan* P = reinterpret_cast<Plan*>(plan);
  cudaStreamSynchronize(P->stream);
  free_plan(P);
  return GBDLT_OK;
}

int gbdlt_plan_profile(gbdlt_plan plan, int mode) {
  if (!plan || mode < 0 || mode > 2) return GBDLT_ERR_INVALID_ARG;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (!P.prof) {
    P.prof = new (std::nothrow) Profiler();
    if (!P.prof) return GBDLT_ERR_OOM;
    P.prof->ev.resize(1024);
    for (cudaEvent_t& e : P.prof->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return GBDLT_ERR_CUDA;
  }
  Profiler& R = *P.prof;
  prof_flush(P);
  if (mode == 2) {
    R.acc.clear();
    return GBDLT_OK;
  }
  R.on = mode == 1;
  R.anchored = false;
  if (R.on) {
    if (cudaEventRecord(R.ev[0], P.stream) != cudaSuccess) return GBDLT_ERR_CUDA;
    R.anchored = true;
  }
  return GBDLT_OK;
}

int64_t gbdlt_plan_profile_read(gbdlt_plan plan, char* buf, int64_t len) {
  if (!plan || len < 0 || (len > 0 && !buf)) return GBDLT_ERR_INVALID_ARG;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  std::string s;
  if (P.prof) {
    prof_flush(P);
    char line[256];
    for (const auto& kv : P.prof->acc) {
      std::snprintf(line, sizeof(line), "%s %lld %.6f %.6e %.6e\n", kv.first.c_str(),
                    (long long)kv.second.count, kv.second.ms, kv.second.flops, kv.second.bytes);
      s += line;
    }
  }
  if (len > 0) {
    const size_t n = std::min<size_t>(s.size(), (size_t)len - 1);
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return (int64_t)s.size();
}

int gbdlt_plan_set_stream(gbdlt_plan plan, void* cuda_stream) {
  if (!plan) return GBDLT_ERR_INVALID_ARG;
  reinterpret_cast<Plan*>(plan)->stream = (cudaStream_t)cuda_stream;
  return GBDLT_OK;
}

int gbdlt_plan_set_node_iterations(gbdlt_plan plan, int max_iter) {
  if (!plan || max_iter < 0 || max_iter > kNodeIterMax) return GBDLT_ERR_INVALID_ARG;
  reinterpret_cast<Plan*>(plan)->node_iter_max = max_iter;
  return GBDLT_OK;
}

int gbdlt_plan_sync(gbdlt_plan plan) {
  if (!plan) return GBDLT_ERR_INVALID_ARG;
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (P->nodes_pending) {
    // a deferred node refresh runs now, so that its status is reported
    P->nodes_pending = false;
    if (int st = launch_legpts(*P, P->CN)) return st;
  }
  if (cudaStreamSynchronize(P->stream) != cudaSuccess) return GBDLT_ERR_CUDA;
  int hs = 0, hi = 0;
  if (cudaMemcpy(&hs, P->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GBDLT_ERR_CUDA;
  // the chain of a plan for N that is not a power of two runs on its inner plan
  if (P->inner && cudaMemcpy(&hi, P->inner->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  if (hi) cudaMemset(P->inner->status, 0, sizeof(int));
  hs |= hi;
  if (hs) {
    cudaMemset(P->status, 0, sizeof(int));
    if (hs & 1) return GBDLT_ERR_NOT_CONVERGED;
    if (hs & 2) return GBDLT_ERR_CUDA;  // an asynchronous tile copy did not complete in time
  }
  return check_launch();
}

int gbdlt_plan_set_wait_limit(gbdlt_plan plan, int64_t sm_cycles) {
  if (!plan || sm_cycles < 0 || sm_cycles > (1ll << 32)) return GBDLT_ERR_INVALID_ARG;
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (P->tma_wait == sm_cycles) return GBDLT_OK;
  // replayed chains hold the limit they were captured with
  if (P->graphs) {
    if (cudaStreamSynchronize(P->graphs->s) != cudaSuccess) return GBDLT_ERR_CUDA;
    free_graphs(P);
  }
  P->tma_wait = sm_cycles;
  if (P->inner) P->inner->tma_wait = sm_cycles;
  return GBDLT_OK;
}

int gbdlt_plan_set_fft_staging(gbdlt_plan plan, int enable) {
  if (!plan || (enable != 0 && enable != 1)) return GBDLT_ERR_INVALID_ARG;
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (P->no_tma == (enable == 0)) return GBDLT_OK;
  // replayed chains hold the kernels they were captured with
  if (P->graphs) {
    if (cudaStreamSynchronize(P->graphs->s) != cudaSuccess) return GBDLT_ERR_CUDA;
    free_graphs(P);
  }
  P->no_tma = enable == 0;
  if (P->inner) P->inner->no_tma = enable == 0;
  return GBDLT_OK;
}

int gbdlt_plan_set_fft_mix(gbdlt_plan plan, int mode) {
  if (!plan || mode < 0 || mode > 2) return GBDLT_ERR_INVALID_ARG;
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (P->fft_mix == mode) return GBDLT_OK;
  // replayed chains hold the launches they were captured with
  if (P->graphs) {
    if (cudaStreamSynchronize(P->graphs->s) != cudaSuccess) return GBDLT_ERR_CUDA;
    free_graphs(P);
  }
  P->fft_mix = mode;
  if (P->inner) P->inner->fft_mix = mode;
  return GBDLT_OK;
}

int gbdlt_plan_get_params(gbdlt_plan plan, gbdlt_params* out) {
  if (!plan || !out) return GBDLT_ERR_INVALID_ARG;
  Plan* P = reinterpret_cast<Plan*>(plan);
  fill_public(P->p, P->ws_bytes, out);
  return GBDLT_OK;
}

int gbdlt_legpts(gbdlt_plan plan, double* x, double* theta, double* w, double* dtheta) {
  if (!plan) return GBDLT_ERR_INVALID_ARG;
  Plan& P = *reinterpret_cast<Plan*>(plan);
  if (!x && !theta && !w && !dtheta) {
    // nothing to copy out: the node kernel runs with the next call that reads the
    // nodes (or at gbdlt_plan_sync)
    P.nodes_pending = true;
    return GBDLT_OK;
  }
  P.nodes_pending = false;
  int st = launch_legpts(P, P.CN);
  if (st) return st;
  const size_t bytes = sizeof(double) * (size_t)P.p.N;
  if (x && cudaMemcpyAsync(x, P.x, bytes, cudaMemcpyDeviceToDevice, P.stream) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  if (theta && cudaMemcpyAsync(theta, P.theta, bytes, cudaMemcpyDeviceToDevice, P.stream) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  if (w && cudaMemcpyAsync(w, P.w, bytes, cudaMemcpyDeviceToDevice, P.stream) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  if (dtheta) {
    st = launch_dtheta(P, dtheta);
    if (st) return st;
  }
  return GBDLT_OK;
}

int gbdlt_leg2cheb(gbdlt_plan p, const void* c, void* chat, int64_t batch) {
  return run_op(p, OP_L2C, c, chat, batch);
}
int gbdlt_leg2cheb_t(gbdlt_plan p, const void* y, void* out, int64_t batch) {
  return run_op(p, OP_L2C_T, y, out, batch);
}
int gbdlt_chebeval(gbdlt_plan p, const void* chat, void* f, int64_t batch) {
  return run_op(p, OP_CHEB, chat, f, batch);
}
int gbdlt_chebeval_t(gbdlt_plan p, const void* g, void* out, int64_t batch) {
  return run_op(p, OP_CHEB_T, g, out, batch);
}
int gbdlt_dlt(gbdlt_plan p, const void* c, void* f, int64_t batch) { return run_op(p, OP_DLT, c, f, batch); }
int gbdlt_dlt_t(gbdlt_plan p, const void* g, void* out, int64_t batch) {
  return run_op(p, OP_DLT_T, g, out, batch);
}
int gbdlt_idlt(gbdlt_plan p, const void* f, void* c, int64_t batch) { return run_op(p, OP_IDLT, f, c, batch); }
int gbdlt_idlt_t(gbdlt_plan p, const void* g, void* out, int64_t batch) {
  return run_op(p, OP_IDLT_T, g, out, batch);
}

const char* gbdlt_status_string(int s) {
  switch (s) {
    case GBDLT_OK: return "ok";
    case GBDLT_ERR_INVALID_ARG: return "invalid argument";
    case GBDLT_ERR_UNSUPPORTED_N: return "unsupported N (power of two, 1..2^24)";
    case GBDLT_ERR_CUDA: return "CUDA error";
    case GBDLT_ERR_OOM: return "device allocation failed";
    case GBDLT_ERR_NOT_CONVERGED: return "node iteration did not converge";
    case GBDLT_ERR_UNIMPLEMENTED: return "unimplemented";
  }
  return "unknown status";
}

uint64_t gbdlt_launch_count(void) { return g_launches.load(); }
uint64_t gbdlt_device_alloc_count(void) { return g_allocs.load(); }

}  // extern "C"
