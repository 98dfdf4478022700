// Internal declarations of the gbdlt CUDA library: plan layout, device
// arithmetic helpers and kernel launchers.  Every launcher enqueues on the
// plan's stream and bumps the library's launch counter.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <vector>

#include "gbdlt.h"

namespace gbdlt {

// ---------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// float-float scalar: value hi + lo (|lo| <= ulp(hi)/2 after normalisation), the
// arithmetic of the FFTs of mid-sized terms in FP64 plans, run on the FP32 pipe
// (64 times the FP64 rate on GB300) with about 2^-47 relative error per
// operation and the exponent range of float.  Operations are explicitly rounded
// so nothing is contracted.  Additions use the cheap form (TwoSum of the heads,
// tails added), whose error is about 2^-47 (|a| + |b|): the transforms need
// norm-wise accuracy, not accuracy relative to each cancelling sum.
struct ffd {
  float hi, lo;
  ffd() = default;
  __host__ __device__ constexpr ffd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr ffd(int v) : hi((float)v), lo(0.f) {}
  // compile-time constants only (two roundings of a double literal)
  __host__ __device__ constexpr ffd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};
__device__ __forceinline__ ffd ff_norm(float s, float e) {
  const float t = __fadd_rn(s, e);
  return ffd(t, __fsub_rn(e, __fsub_rn(t, s)));
}
__device__ __forceinline__ ffd operator+(ffd a, ffd b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return ff_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ffd operator-(ffd a) { return ffd(-a.hi, -a.lo); }
__device__ __forceinline__ ffd operator-(ffd a, ffd b) { return a + (-b); }
__device__ __forceinline__ ffd operator*(ffd a, ffd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_norm(p, e);
}
__device__ __forceinline__ ffd& operator+=(ffd& a, ffd b) {
  a = a + b;
  return a;
}
// a.x b.x - a.y b.y (sign = -1) or a.x b.y + a.y b.x style dot of two products,
// one normalisation: p1 + sign p2 with both product errors carried in the tail
__device__ __forceinline__ ffd ff_dot2(ffd a1, ffd b1, ffd a2, ffd b2, float sign) {
  const float p1 = __fmul_rn(a1.hi, b1.hi);
  float e1 = __fmaf_rn(a1.hi, b1.hi, -p1);
  e1 = __fmaf_rn(a1.hi, b1.lo, e1);
  e1 = __fmaf_rn(a1.lo, b1.hi, e1);
  const float h2 = sign * a2.hi, l2 = sign * a2.lo;  // exact
  const float p2 = __fmul_rn(h2, b2.hi);
  float e2 = __fmaf_rn(h2, b2.hi, -p2);
  e2 = __fmaf_rn(h2, b2.lo, e2);
  e2 = __fmaf_rn(l2, b2.hi, e2);
  const float s = __fadd_rn(p1, p2);
  const float bb = __fsub_rn(s, p1);
  const float es = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
  return ff_norm(s, __fadd_rn(es, __fadd_rn(e1, e2)));
}
struct alignas(16) ffc {
  ffd x, y;
};

template <typename T>
struct Cx;
template <>
struct Cx<double> {
  using type = double2;
};
template <>
struct Cx<float> {
  using type = float2;
};
template <>
struct Cx<ffd> {
  using type = ffc;
};
template <typename T>
constexpr bool is_f64 = false;
template <>
constexpr bool is_f64<double> = true;
template <typename T>
constexpr bool is_f32 = false;
template <>
constexpr bool is_f32<float> = true;
template <typename T>
using C2 = typename Cx<T>::type;

template <typename T>
__host__ __device__ __forceinline__ C2<T> mk(T a, T b) {
  C2<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  if constexpr (std::is_same<T, ffd>::value) {
    return mk<T>(ff_dot2(a.x, b.x, a.y, b.y, -1.f), ff_dot2(a.x, b.y, a.y, b.x, 1.f));
  } else {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }
}
template <typename T>
__device__ __forceinline__ C2<T> cconj(C2<T> a) {
  return mk<T>(a.x, -a.y);
}
// multiply by +i (DIR > 0) or -i (DIR < 0)
template <typename T, int DIR>
__device__ __forceinline__ C2<T> cmul_i(C2<T> a) {
  return DIR > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}
template <typename T>
__device__ __forceinline__ C2<T> to_c(double2 a) {
  return mk<T>((T)a.x, (T)a.y);
}

// ---------------------------------------------------------------------------
// double-double helpers for the node kernel (error-free transformations with
// explicitly rounded operations so the compiler cannot contract them)
// ---------------------------------------------------------------------------
struct ddv {
  double hi, lo;
};
__device__ __forceinline__ ddv dd_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ddv dd_quick(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ ddv dd_add(ddv a, ddv b) {
  ddv s = dd_two_sum(a.hi, b.hi);
  ddv t = dd_two_sum(a.lo, b.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = dd_quick(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return dd_quick(s.hi, s.lo);
}
__device__ __forceinline__ ddv dd_mul(ddv a, ddv b) {
  double p = __dmul_rn(a.hi, b.hi);
  double e = __fma_rn(a.hi, b.hi, -p);
  e = __fma_rn(a.hi, b.lo, e);
  e = __fma_rn(a.lo, b.hi, e);
  return dd_quick(p, e);
}
__device__ __forceinline__ ddv dd_mul_d(ddv a, double b) {
  double p = __dmul_rn(a.hi, b);
  double e = __fma_rn(a.hi, b, -p);
  e = __fma_rn(a.lo, b, e);
  return dd_quick(p, e);
}
// a / b for doubles, correct to dd precision
__device__ __forceinline__ ddv dd_div_dd(double a, double b) {
  double q = __ddiv_rn(a, b);
  double r = __fma_rn(-q, b, a);
  return dd_quick(q, __ddiv_rn(r, b));
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
// per-row factors of the asymptotic expansion (stages.cu)
struct alignas(32) RowAR {
  double ax, ay, rx, ry;
};

struct Band {
  int64_t ns;  // columns n >= ns use the asymptotic expansion
  int64_t ka;  // rows [ka, kb) and [N-kb, N-ka)
  int64_t kb;
};

// Two-level twiddle table for e^{2 pi i e / B}, 0 <= e < B:
// value = hi[e >> 12] * lo[e & 4095].
struct Twiddle2 {
  double2* lo = nullptr;  // 4096 entries
  double2* hi = nullptr;  // max(1, B / 4096) entries
  int64_t B = 0;
};

struct Params {
  int64_t N = 0;
  int prec = GBDLT_FP64;
  double eps = 0;
  int L = 1;
  int M = 0;
  int K = 0;
  std::vector<Band> bands;
  int seg = 512;
  int64_t rec_steps = 0;
  double flops_dlt = 0, bytes_dlt = 0, bytes_idlt = 0;
  int method = GBDLT_METHOD_FAST;  // what gbdlt_dlt/idlt(_t) run (resolved, never AUTO)
  bool fast = true;                // N is a power of two: the FFT-based chains exist
  int64_t direct_steps = 0;        // half-row recurrence steps of one direct transform
  int64_t head = 0;                // columns n < head come from the dense block M[0:head, 0:head]
  int Mh = 0;                      // expansion terms whose band FFTs run in the plan's precision;
                                   // terms Mh..M-1 of an FP64 plan run in FP32
  int M64 = 0;                     // of those, terms M64..Mh-1 of an FP64 plan run in float-float
  int Lff = 0;                     // Taylor terms l >= Lff of an FP64 plan run in float-float
  int64_t grid = 0;                // fast path: length G of the Chebyshev grid and FFTs (N for a
                                   // power of two, the next power of two otherwise); 0: direct only
  double taylor_b = 0.83845;       // bound on |n dtheta_k| behind L and Lff (Corollary 2.4)
};

// Direct method limits: largest N a direct plan accepts, and the largest
// power-of-two N that GBDLT_METHOD_AUTO sends to the direct method.
constexpr int64_t kDirectMax = 1 << 16;
constexpr int64_t kDirectAuto = 256;
// largest dense head block a fast plan uses (h^2/4 terms per transform)
// Mixed FP64 / float-float Taylor FFT launches pay from this length up
// (GB300, FP64 step: 5.56 -> 5.55 ms at 2^20, 26.7 -> 26.3 ms at 2^22); below
// it the two-stream launches are faster (2^18: 1.76 against 1.88 ms), the mixed
// grid being too short to keep two FP64 thread blocks on every SM.
constexpr int64_t kFftMixMinN = 1 << 20;
constexpr int64_t kHeadMax = 1 << 16;
// largest head block whose products an FP64 plan stores (h^2/4 doubles: 2.1 GB)
constexpr int64_t kHeadTabMax = 1 << 15;

// Fills Params from (N, prec, eps, method): Taylor terms, asymptotic terms, bands
// and the method the plan runs.  taylor_b bounds |n dtheta_k| over the columns
// and rows the Taylor step serves (0.83845 for the Legendre nodes against the
// cheb1 grid of the same N, Lemma 2.3).
int derive_params(int64_t N, int prec, double eps, int method, Params* p, double taylor_b = 0.83845);
// Host table of C_n = sqrt(4/pi) Gamma(n+1)/Gamma(n+3/2), n = 0..N (double-double recurrence).
std::vector<double> cn_table(int64_t N);

struct RecLayout {
  int64_t H = 0;              // half rows (ceil(N / 2); row H-1 is its own mirror for odd N)
  int64_t half_steps = 0;     // recurrence steps over all half rows
  int S = 512;                // segment length
  int j0 = 0;                 // first segment run (columns below j0 S are the dense head's)
  int64_t nseg_total = 0;     // sum over half rows of nseg(k)
  int64_t n_long = 0;         // rows [0, n_long) have nseg > 64
  int64_t nblocks = 0;        // row blocks of 256 half rows
  int64_t ncta = 0;           // (row block, segment) pairs
  int64_t tbuf_total = 0;     // transposed partial buffer length
  int64_t n_heavy = 0;        // columns n below the cuts of more than 32 row blocks
  // device arrays
  int32_t* cut = nullptr;     // [H] recurrence cut per half row
  int64_t* poff = nullptr;    // [H] offset of row k's segments
  int32_t* cta_rb = nullptr;  // [ncta]
  int32_t* cta_j = nullptr;   // [ncta] first segment j, A - 1 << 16, q - 1 << 20 (rec.cu, RecTask)
  // forward recurrence: the (segment, row) pairs of each row block packed into
  // full warps (rec.cu, k_rec_fwd): nfw warps of fwpc per CTA, per warp its row
  // block, per lane its row within the block | segment << 8 (-1: none)
  int64_t nfw = 0;
  int fwpc = 8;
  int32_t* fw_rb = nullptr;   // [nfw]
  int32_t* fw_lane = nullptr; // [32 nfw]
  // transposed recurrence of fast layouts (rec.cu, k_rec_tp): ntw warps of twpc
  // per CTA over the (row, segment) pairs ordered by segment; per lane its half
  // row and slot (-1: none), per slot its segment and S column sums per batch
  // item, per segment j >= j0 its first slot (tsegs + 1 entries)
  int64_t ntw = 0;
  int twpc = 8;
  int64_t tslots = 0;
  int tsegs = 0;
  int32_t* tw_k = nullptr;       // [32 ntw]
  int32_t* tw_slot = nullptr;    // [32 ntw]
  int32_t* tslot_j = nullptr;    // [tslots]
  int32_t* tseg_begin = nullptr; // [tsegs + 1]
  double* tpart = nullptr;       // [batch][tslots][S]
  int64_t* toff = nullptr;    // [nblocks] offset of row block partials (length nseg_max*S)
  int32_t* bcutmax = nullptr; // [nblocks] nseg_max(rb) * S (partial array length)
  double* xm1 = nullptr;      // [H] x_k - 1 of the rows (cheb1 grid, or Legendre nodes)
  double2* state = nullptr;   // [nseg_total] (P, D) at segment starts
  double2* part = nullptr;    // [nseg_total] forward partial sums (E, O)
  double* tbuf = nullptr;     // [tbuf_total] transposed partial sums
  double* rscratch = nullptr; // [ceil(nblocks/64)][n_heavy] chunk sums of the transposed reduction
};

// Newton iterations a node may take before the node kernels flag it as not
// converged (the cap a plan uses unless gbdlt_plan_set_node_iterations lowers it)
constexpr int kNodeIterMax = 24;

struct Plan {
  Params p;
  int device = 0;
  cudaStream_t stream = nullptr;
  // nodes (double)
  double* theta = nullptr;
  double* x = nullptr;
  double* w = nullptr;
  double* tN = nullptr;  // N * dtheta_k
  // tables
  double* Cn = nullptr;     // [N+1]
  double* ra = nullptr;     // (2n+1)/(n+1)
  double* rb = nullptr;     // n/(n+1)
  float2* ra_ff = nullptr;  // the same as float-float (hi, lo), for the FP32 form
  float2* rb_ff = nullptr;
  double2* tw4096 = nullptr;
  Twiddle2 twN, tw4N;
  // the same tables rounded to float, used by the FP32 form (no FP64 work there)
  float2* tw4096f = nullptr;
  float2 *twNf_lo = nullptr, *twNf_hi = nullptr, *tw4Nf_lo = nullptr, *tw4Nf_hi = nullptr;
  // FP64 FFT tables: e^{2 pi i e/N} for every e < N (the four-step twiddle; FP64
  // plans with N > 4096 only), and the cosine/tangent form of e^{+-2 pi i e/4096}
  // used by the fused radix-4 layers ([2 directions][4096][sx, sy, t, swap])
  double2* twfull = nullptr;
  double2* lf_tab = nullptr;
  // the same e^{2 pi i j/4096} and e^{2 pi i e/N} as float-float pairs, for the
  // float-float FFTs of FP64 plans
  ffc* tw4096_ff = nullptr;
  ffc* twfull_ff = nullptr;
  // FP64 stage tables: C_n h_{m,n} ([Mh][N], the asymptotic expansion's column
  // weights of the FP64 terms) and per cheb1 row {alpha_k, rho_k} (the expansion's
  // row factors)
  double* Hnm = nullptr;
  RowAR* row_ar = nullptr;
  // dense head block: Lam'_j = sqrt(2/pi) Gamma(j+1/2)/Gamma(j+1), j < head
  double* head_lam = nullptr;
  float* head_lamf = nullptr;
  // FP64 plans with head <= kHeadTabMax: the products M_{k,n} of the head block,
  // row k (n = k, k+2, ..., < head) from offset head_off[k] (head.cu)
  double* head_tab = nullptr;
  int64_t* head_off = nullptr;
  // the same products column by column (column n holds rows k = n mod 2, ...,
  // n from offset head_offT[n]): the transposed block reads them contiguously
  double* head_tabT = nullptr;
  int64_t* head_offT = nullptr;
  // FP32 plans with head > kHeadMM: the register-blocked head kernels (head.cu):
  // Lam' with kHeadPad zeros on both sides, their warp tasks (forward, then
  // transposed) and the per-item chunk partials
  float* head_lamp = nullptr;
  int4* head_tasks = nullptr;
  int head_ntask_f = 0, head_ntask_t = 0;
  double* head_part = nullptr;
  int64_t head_part_n = 0;  // doubles per batch item
  int head_rbc = 0;         // reduction indices per task
  int64_t* band_dev = nullptr;  // [3K] ns, ka, kb
  RecLayout rec;    // recurrence region of the fast path (cheb1 rows)
  RecLayout drec;   // every row and column at the Legendre nodes (direct method)
  bool has_direct = false;
  // workspace (element type = plan precision)
  void* bufA = nullptr;
  void* bufB = nullptr;
  int64_t nfft_max = 0;  // FFT vectors per transform (per batch item)
  // the FP32 band vectors of an FP64 plan ([item][band][term Mh..M-1][N] float2)
  void* bufA32 = nullptr;
  void* bufB32 = nullptr;
  // the float-float band vectors of an FP64 plan ([item][band][term M64..Mh-1][N] ffc)
  void* bufAff = nullptr;
  void* bufBff = nullptr;
  // their power-of-two scales: per (band, term) exponents [2][K][M] (forward,
  // transposed) and per batch item the bits of max |chain input|
  int* b32exp = nullptr;
  unsigned long long* absmax = nullptr;
  float* H32 = nullptr;  // [M - Mh][N] C_n h_{m,n} 2^{e_{K-1,m}} of the FP32 terms (stages.cu)
  ffd* Hff = nullptr;    // [Mh - M64][N] the same for the float-float terms
  int prune_bands = 0;   // leading bands whose FFTs are pruned to their row windows
  int prune_R = 0;       // window half-width of those bands (bins)
  int64_t bcap = 1;      // batch items one pass over the workspace holds
  void* v = nullptr;     // [N]
  void* chat = nullptr;  // [N]
  void* z = nullptr;     // [N]
  void* tmp = nullptr;   // [N]
  void* tmp2 = nullptr;  // [N]
  int* status = nullptr; // device status word
  int node_iter_max = kNodeIterMax;  // Newton iterations a node may take (legpts.cu)
  // FP32 FFT passes without the TMA-staged kernels (fft.cu): the default of FP64
  // plans, whose FP32 transforms run on the side stream beside FP64 kernels and
  // there leave more room to them as ordinary (non-persistent) grids
  bool no_tma = false;
  // FP64 plans: the FP64 and float-float FFTs of the Taylor stages in one mixed
  // pair of launches (fft.cu, launch_fft_mix) instead of two streams: 0 never,
  // 1 at N >= kFftMixMinN (the default), 2 at every four-step length
  int fft_mix = 1;
  long long tma_wait = 1ll << 32;  // SM cycles a staged pass waits for a tile copy
  void* arena = nullptr; // single device allocation holding everything above
  size_t ws_bytes = 0;
  double CN = 0;         // C_N for the node kernel
  // side stream for FP32-pipe work (float-float and FP32 transforms) that runs
  // beside FP64 work of the same chain; created on first use
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool side_broken = false;  // creation failed: everything on the plan stream
  struct Profiler* prof = nullptr;  // per-kernel event timing (off unless enabled)
  struct GraphCache* graphs = nullptr;  // replayed transform chains (plan.cu)
  // gbdlt_legpts without outputs defers the node kernel to the next call that
  // reads the nodes, where it runs as a branch beside that chain's first stages
  // (plan.cu, nodes_start / nodes_ready)
  bool nodes_pending = false;
  bool node_branch_open = false;  // the branch is in flight: readers wait on node_join
  cudaStream_t node_s = nullptr;
  cudaEvent_t node_fork = nullptr, node_join = nullptr;
  // N not a power of two (grid.cu): the fast path is the chain of `inner`, a plan
  // on the power-of-two grid G > N, fed with inputs zero-padded to G; this plan
  // keeps the N-point rule (and the direct method's layout)
  Plan* inner = nullptr;
  void* rg_in = nullptr;   // [bcap][G] padded inputs
  void* rg_out = nullptr;  // [bcap][G] chain outputs before truncation to N
  // on an inner plan: the rows are those of other rules (N-point Gauss-Legendre
  // rules with N <= G) placed on this plan's grid, one rule per batch item
  const struct GridRule* rg_rules = nullptr;  // device [rules]; null: this plan's own nodes
  const int32_t* rg_item = nullptr;  // device [items] rule of each item (null: rule 0 for all)
  int64_t rg_item0 = 0;              // first item of the pass run_chain is running
  int64_t rg_nmax = 0;               // longest rule (launch sizes)
  void* rg_g = nullptr;              // [bcap][G] rows summed onto their grid points
  struct GridRules* rg_own = nullptr;  // rules this plan owns (a plan for N not a power of two)
};

// An N-point rule on a grid of G >= N points (grid.cu): row k's nearest grid
// point j[k], its offset t[k] = G (theta_k - (j[k] + 1/2) pi / G), the first row
// kf[jj] of grid point jj (jj = 0..G), and the rule's weights.
struct GridRule {
  int64_t n;
  const int32_t* j;
  const double* t;
  const int32_t* kf;
  const double* w;
};

// Taylor pairs whose FFTs run in the plan's precision: pair p holds terms
// 2p + (inc0 ? 0 : 2) and 2p + 1; it runs in float-float when both are >= Lff
inline int taylor_p64(const Params& p, int inc0, int npair) {
  const int lo = p.Lff;
  const int q = inc0 ? (lo + 1) / 2 : lo / 2;  // first pair whose smaller term is >= Lff
  return q < npair ? q : npair;
}

// twiddle tables in the precision T of a transform
template <typename T>
struct TwT {
  const C2<T>* t4096;  // e^{2 pi i j / 4096}
  const C2<T>* nlo;    // e^{2 pi i e / N}, two-level
  const C2<T>* nhi;
  const C2<T>* flo;    // e^{2 pi i e / (4N)}, two-level
  const C2<T>* fhi;
  const C2<T>* full;   // e^{2 pi i e / N}, one entry per e (FP64 only, else null)
  const double2* lf;   // cosine/tangent twiddles (FP64 only, else null)
};
inline TwT<double> tw_tables(const Plan& P, double) {
  return {P.tw4096, P.twN.lo, P.twN.hi, P.tw4N.lo, P.tw4N.hi, P.twfull, P.lf_tab};
}
inline TwT<float> tw_tables(const Plan& P, float) {
  return {P.tw4096f, P.twNf_lo, P.twNf_hi, P.tw4Nf_lo, P.tw4Nf_hi, nullptr, nullptr};
}
inline TwT<ffd> tw_tables(const Plan& P, ffd) {
  return {P.tw4096_ff, nullptr, nullptr, nullptr, nullptr, P.twfull_ff, nullptr};
}

// Before a kernel that reads the plan's nodes (tN, w, theta, x): the plan stream
// waits for a node branch in flight (a deferred gbdlt_legpts), if any.
int nodes_ready(Plan& P);

// plan lifecycle and the operator dispatch shared by the C ABI and the batch
// executor; max_batch > 0 limits the batch items one workspace pass holds
// want_direct also builds the direct layout for a fast plan (the batch autotuner
// times both methods on one plan)
int plan_create_impl(int64_t N, int prec, double eps, int method, cudaStream_t stream, int64_t max_batch,
                     int want_direct, Plan** out);
// a plan holding only the N-point rule (nodes, weights, N dtheta): the rules of
// a batch's grid groups
int plan_create_nodes(int64_t N, int prec, cudaStream_t stream, Plan** out);
// a fast plan for the power-of-two G whose Taylor step serves rows with
// |n dtheta| <= taylor_b (rules placed on its grid)
int plan_create_grid(int64_t G, int prec, double eps, double taylor_b, cudaStream_t stream, int64_t max_batch,
                     Plan** out);
void free_plan(Plan* P);
enum Op { OP_L2C, OP_L2C_T, OP_CHEB, OP_CHEB_T, OP_DLT, OP_DLT_T, OP_IDLT, OP_IDLT_T };
int run_op(gbdlt_plan plan, int op, const void* in, void* out, int64_t batch);
// the same with the method of the four transforms given (GBDLT_METHOD_FAST / _DIRECT)
int run_op_method(gbdlt_plan plan, int op, int method, const void* in, void* out, int64_t batch);

// ---------------------------------------------------------------------------
// launch bookkeeping
// ---------------------------------------------------------------------------
void count_launch(int n = 1);
int check_launch();  // GBDLT_OK or GBDLT_ERR_CUDA after a launch
// cudaMalloc that counts the library's device allocations (gbdlt_device_alloc_count)
cudaError_t dev_malloc(void** p, size_t bytes);
// Counts one launch and, when the plan's profiler is on, records an event after
// it tagged with the kernel name and its algorithmic flops and bytes.
void launched(Plan& P, const char* name, double flops, double bytes);

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
// tables.cu
int launch_twiddle_init(Plan& P);
// fft.cu: the FP64 transform tables (twfull, lf_tab)
int launch_fft_tables_init(Plan& P);
// stages.cu: the FP64 stage tables (Hnm, row_ar)
int launch_stage_tables_init(Plan& P);
// legpts.cu
// blocks_per_sm > 0: a grid of that many blocks per SM strides over the nodes
// (the node kernel as a branch beside other kernels leaves room on every SM)
int launch_legpts(Plan& P, double CN, int blocks_per_sm = 0);
int launch_dtheta(Plan& P, double* out);  // out_k = t_k / N
// fft.cu: in-place batched FFT of length N, sign DIR (+1: e^{+2 pi i nk/N}).
// Input in `a`; result in `a` when N <= 4096, else in `b` (returned pointer).
template <typename T>
void* launch_fft(Plan& P, void* a, void* b, int64_t nvec, int dir);
// the FP64 vectors a64 (nv64) and the float-float vectors aff (nvff) of one
// stage, both of length N > 4096, in one pair of launches whose CTAs alternate
// between the two kinds (separate pipes on GB300); results in b64 and bff
void launch_fft_mix(Plan& P, void* a64, void* b64, int64_t nv64, void* aff, void* bff, int64_t nvff, int dir);
// the K*M band FFTs of nb items (vectors [item][band][term]); bands
// [0, prune_bands) read only the windows of their rows (transposed = 0: forward
// chain, outputs pruned; 1: transposed chain, inputs pruned)
template <typename T>
void* launch_fft_bands(Plan& P, void* a, void* b, int64_t nb, int dir, int transposed, int terms);
// rec.cu
int launch_rec_state_init(Plan& P, RecLayout& L);
template <typename T>
int launch_rec_forward(Plan& P, RecLayout& L, const T* c, T* vrec, int64_t nb);
template <typename T>
int launch_rec_transpose(Plan& P, RecLayout& L, const T* z, T* out, int64_t nb,
                         const double* zw = nullptr, int scale_out = 0);
// x_k - 1 of the cheb1 rows (fast path) or of the Legendre nodes (direct method)
int launch_rec_xm1(Plan& P, RecLayout& L, int legendre);
// Many small direct-method transforms in one persistent launch (uneven batches):
// the groups' transforms, `count` vectors of length N each, contiguous from
// `in` / `out`, all of one direction (0: DLT, 1: IDLT).  Only plans whose direct
// layout is one CTA (direct_fusable) take part; results are bitwise those of
// run_op_method with GBDLT_METHOD_DIRECT.
// grid.cu: rules on a power-of-two grid.  grid_rules_create places the rules of
// the given node plans (their theta, N dtheta and weights) on a grid of G
// points and checks that no grid point holds more than two rows; the device
// table has one GridRule per node plan, in order.  grid_bound is the bound b on
// |n dtheta| over the rules (Corollary 2.4): (N-1) pi / (2G) for N < G, 0.83845
// for N = G.  grid_attach gives inner plan I the rules `R` (I.rg_*), with
// `item` the rule of each batch item (device, or null for rule 0).
// launch_grid_pad copies [nb][N] into [nb][G] with zeros past N,
// launch_grid_cut the first N of each [G] row back; launch_grid_scatter sums the
// rows (times w_k when use_w) onto their grid points (the l = 0 Taylor term of
// the transposed chain).
struct GridRules;
double grid_bound(int64_t N, int64_t G);
int grid_rules_create(int64_t G, const std::vector<Plan*>& nodes, cudaStream_t s, GridRules** out);
void grid_rules_free(GridRules* r);
size_t grid_rules_bytes(const GridRules* r);
int grid_attach(Plan& I, GridRules* R, const int32_t* item, bool own);
template <typename T>
int launch_grid_pad(Plan& P, const T* in, T* out, int64_t N, int64_t G, int64_t nb);
template <typename T>
int launch_grid_cut(Plan& P, const T* in, T* out, int64_t N, int64_t G, int64_t nb);
template <typename T>
int launch_grid_scatter(Plan& I, const T* g, int use_w, T* out, int64_t nb);

struct DirectGroupRef {
  Plan* plan;
  int64_t count;
  const void* in;
  void* out;
};
struct DirectMulti;
bool direct_fusable(const Plan& P);
int direct_multi_create(const std::vector<DirectGroupRef>& groups, int prec, int dir, DirectMulti** out);
int direct_multi_launch(DirectMulti* d, cudaStream_t s);
int64_t direct_multi_jobs(const DirectMulti* d);
void direct_multi_free(DirectMulti* d);
// stages.cu (prologues / epilogues)
// band vectors of terms m < M64 in U / Y / F (precision T), of terms
// M64 <= m < Mh in Uff / Yff / Fff (float-float) and of terms m >= Mh in U32 /
// Y32 / F32 (FP32); the last two exist in FP64 plans only
template <typename T>
int launch_l2c_pro(Plan& P, const T* c, C2<T>* U, ffc* Uff, float2* U32, int64_t nb);
// max |x| per batch item into P.absmax (FP64 plans with FP32 band vectors)
template <typename T>
int launch_absmax(Plan& P, const T* x, int64_t nb);
template <typename T>
int launch_l2c_epi(Plan& P, const C2<T>* Y, const ffc* Yff, const float2* Y32, const T* vrec, T* v, int64_t nb);
template <typename T>
int launch_a4_pro(Plan& P, const T* v, C2<T>* U, int64_t nb);
// hb != null: add the head block's written result (launch_head_fwd with hout)
template <typename T>
int launch_a4_epi(Plan& P, const C2<T>* F, T* chat, int64_t nb, const double* hb = nullptr);
template <typename T>
int launch_fcs_pro(Plan& P, const T* a, C2<T>* U, int scale_d, int64_t nb);
// Taylor pairs: p < taylor_p64 in U / Y / F (precision T, [item][P64][N]); with
// Uff / Yff / Fff given (FP64 plans), pairs p >= P64 there in float-float
template <typename T>
int launch_tay_pro(Plan& P, const T* chat, C2<T>* U, ffc* Uff, int inc0, int npair, int64_t nb);
template <typename T>
int launch_tay_epi(Plan& P, const C2<T>* Y, const ffc* Yff, const T* v, T* f, int inc0, int npair, int64_t nb);
template <typename T>
int launch_tayt_pro(Plan& P, const T* f, int use_w, C2<T>* U, ffc* Uff, int inc0, int npair, int64_t nb);
template <typename T>
int launch_tayt_epi(Plan& P, const C2<T>* F, const ffc* Fff, C2<T>* Q, T* u_out, int inc0, int npair, int64_t nb,
                    int64_t nu = -1);
template <typename T>
int launch_l2ct_pro(Plan& P, const C2<T>* Y, const T* g, int use_w, T* z, C2<T>* U, ffc* Uff, float2* U32,
                    int64_t nb);
// hb != null: add the transposed head block's written result (launch_head_t with hout)
template <typename T>
int launch_l2ct_epi(Plan& P, const C2<T>* F, const ffc* Fff, const float2* F32, const T* rect, T* out, int scale_s,
                    int64_t nb, const double* hb = nullptr);
template <typename T>
int launch_fcs_re_epi(Plan& P, const C2<T>* Y, T* out, int64_t nb);
template <typename T>
int launch_scale(Plan& P, const T* in, T* out, int which, int64_t nb);
// head.cu: the dense head block, chat[0:h] += M[0:h, 0:h] c[0:h], and its
// transpose, out[0:h] += D M[0:h, 0:h]^T y[0:h] (D = diag(n + 1/2) when scale_s)
// With hout given, the block's result is written (double; item stride N sizeof(T)/8
// doubles, so it fits in an N-element buffer of the plan's precision) instead of
// being added; the A4 / transposed leg2cheb epilogues then add it (hb below).
template <typename T>
int launch_head_fwd(Plan& P, const T* c, T* chat, int64_t nb, double* hout = nullptr);
template <typename T>
int launch_head_t(Plan& P, const T* y, T* out, int scale_s, int64_t nb, double* hout = nullptr);
// fills P.head_tab from P.head_lam (plan creation)
int launch_head_tab_init(Plan& P);
// FP32 head blocks above kHeadMM columns run register-blocked warp tasks of 8
// outputs per lane over chunks of *rbc reduction indices; the host side picks
// the chunk, lists the tasks (x, y, z = parity, output block, chunk) of both
// directions and sizes the partial buffer (doubles per batch item)
constexpr int64_t kHeadMM = 2048;
constexpr int kHeadPad = 1536;
void head_rb_tasks(int64_t h, std::vector<int4>& fwd, std::vector<int4>& trn, int64_t* part_n, int* rbc);

}  // namespace gbdlt
