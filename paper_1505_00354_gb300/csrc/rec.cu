// Recurrence region of leg2cheb and of its transpose (Sec. 3; the direct
// three-term recurrence of Sec. 2.4 / Sec. 4.1 applied where the asymptotic
// expansion of P_n(cos theta) is not accurate), and the direct method (the same
// kernels over every column at the Legendre nodes: Eq. (1), and Eq. (2) with the
// weights on the rows and n + 1/2 on the reduction).
//
// A layout (RecLayout) gives per half row k its x_k - 1 and its column cut.  In the
// fast path the rows are the cheb1 points theta_k = (k+1/2)pi/N and row k uses the
// recurrence for columns n < cut(k) (cut = N for the rows nearest theta = 0, pi;
// the band's column cut otherwise); in the direct method the rows are the
// Legendre nodes and every cut is N (for odd N the middle row, x = 0, is its own
// mirror).  Rows k and N-1-k share one recurrence because
// P_n(-x) = (-1)^n P_n(x): with E = sum over even n and O over odd n of c_n P_n(x_k),
//   v_k = E + O,  v_{N-1-k} = E - O.
// The recurrence runs in difference form with x - 1 = -2 sin^2(theta/2) computed
// directly (no cancellation near x = 1, where the plain form loses ~n^2 u):
//   D_{n+1} = [(2n+1)(x-1) P_n + n D_n] / (n+1),   P_{n+1} = P_n + D_{n+1},
//   (P_0, D_0) = (1, 1).
// Each half row's column range is cut into segments of S columns (512; 256 in
// the fast path of FP32 plans); the state (P, D) at every segment start depends
// only on N, so the plan computes it
// once (two basis solutions per segment, then a scan per row) and the transforms
// run every segment independently.  The FP64 kernels carry G_n = D_n / (x - 1)
// instead of D_n, which takes one FP64 instruction less per step (FP64 issue is
// what bounds them on GB300) with the same roundings:
//   G_{n+1} = (2n+1)/(n+1) P_n + n/(n+1) G_n,   P_{n+1} = P_n + (x-1) G_{n+1}
// (one multiply and two fused multiply-adds).  The FP64 form runs the recurrence in FP64;
// the FP32 form runs it in float-float (compensated FP32, ~2^-44 per operation)
// on the FP32 pipe, which is 58 times faster than the FP64 pipe on GB300.
#include <algorithm>
#include <new>
#include <vector>

#include "gbdlt_internal.cuh"

namespace gbdlt {

namespace {

constexpr int RT = 256;  // threads per CTA = half rows per row block

struct RecArgs {
  int64_t N, H;
  int64_t mid;         // the half row that is its own mirror (odd N), else -1
  int S;
  int64_t nblocks;
  int64_t nseg_total;  // batch stride of the segment partials
  int64_t tbuf_total;  // batch stride of the transposed partials
  const int32_t* cut;
  const int64_t* poff;
  const double2* state;
  const int32_t* cta_rb;
  const int32_t* cta_j;
  const int32_t* fw_rb;    // forward warps: row block per warp
  const int32_t* fw_lane;  // forward warps: row | segment << 8 per lane (-1: none)
  int64_t nfw;
  const int32_t* tw_k;        // transposed warps: half row per lane (-1: none)
  const int32_t* tw_slot;     // transposed warps: slot per lane (-1: none)
  const int32_t* tslot_j;     // segment of each slot
  const int32_t* tseg_begin;  // first slot of each segment j >= j0
  int64_t ntw, tslots;
  int tsegs;
  const int64_t* toff;
  const int32_t* maxcut;
  const double* ra;
  const double* rb;
  const float2* raf;
  const float2* rbf;
  const double* xm1;   // [H] x_k - 1
  const double* zw;    // transposed input weights (w_k for the direct IDLT), or null
  int64_t n_heavy;     // columns below the cuts of more than 32 row blocks
  int64_t rchunks;     // chunks of 64 row blocks
  double* rscratch;    // [batch][rchunks][n_heavy] chunk sums
  int scale_out;       // transposed reduction: 1 multiplies out_n by n + 1/2
  int j0;              // first segment run (the dense head block covers n < n_lo)
  int64_t n_lo;        // j0 * S
};

// ---------------------------------------------------------------------------
// float-float arithmetic (compensated FP32) for the FP32 form's recurrence:
// a value is hi + lo with |lo| <= ulp(hi)/2; products use fmaf (TwoProd),
// sums TwoSum; operations are explicitly rounded so nothing is contracted.
// ---------------------------------------------------------------------------
struct ffv {
  float hi, lo;
};
__device__ __forceinline__ ffv ff_quick(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ffv ff_add(ffv a, ffv b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_quick(s, e);
}
__device__ __forceinline__ ffv ff_mul(ffv a, ffv b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_quick(p, e);
}
// the same product left unnormalised (|lo| may exceed half an ulp of hi): for
// operands that go straight into ff_mul or ff_add, whose error-free steps take
// hi and lo as they come and renormalise at the end
__device__ __forceinline__ ffv ff_mul_raw(ffv a, ffv b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}
__device__ __forceinline__ ffv ff_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ ffv ff_ld(const float2 v) { return {v.x, v.y}; }
// Kahan-compensated float accumulator: value = s - c
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

RecArgs rec_args(const Plan& P, const RecLayout& L) {
  RecArgs a;
  a.N = P.p.N;
  a.H = L.H;
  a.mid = (P.p.N & 1) ? L.H - 1 : -1;
  a.S = L.S;
  a.nblocks = L.nblocks;
  a.nseg_total = L.nseg_total;
  a.tbuf_total = L.tbuf_total;
  a.cut = L.cut;
  a.poff = L.poff;
  a.state = L.state;
  a.cta_rb = L.cta_rb;
  a.cta_j = L.cta_j;
  a.fw_rb = L.fw_rb;
  a.fw_lane = L.fw_lane;
  a.nfw = L.nfw;
  a.tw_k = L.tw_k;
  a.tw_slot = L.tw_slot;
  a.tslot_j = L.tslot_j;
  a.tseg_begin = L.tseg_begin;
  a.ntw = L.ntw;
  a.tslots = L.tslots;
  a.tsegs = L.tsegs;
  a.toff = L.toff;
  a.maxcut = L.bcutmax;
  a.xm1 = L.xm1;
  a.zw = nullptr;
  a.scale_out = 0;
  a.n_heavy = L.n_heavy;
  a.rchunks = (L.nblocks + 63) / 64;
  a.rscratch = L.rscratch;
  a.j0 = L.j0;
  a.n_lo = (int64_t)L.j0 * L.S;
  a.ra = P.ra;
  a.rb = P.rb;
  a.raf = P.ra_ff;
  a.rbf = P.rb_ff;
  return a;
}

// x - 1 = -2 sin^2(theta/2) per half row: theta_k = (k+1/2)pi/N (cheb1 grid of
// the fast path) or the Legendre node theta_k (direct method)
__global__ void k_rec_xm1(double* __restrict__ xm1, const double* __restrict__ theta, int64_t H, int64_t N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= H) return;
  const double s = theta ? sin(0.5 * theta[k]) : sinpi((double)(2 * k + 1) / (double)(4 * N));
  xm1[k] = -2.0 * s * s;
}

__device__ __forceinline__ int nseg_of(const RecArgs& R, int64_t k) {
  return (R.cut[k] + R.S - 1) / R.S;
}
// A CTA's work: row block rb and q consecutive segments j, j+1, ..., j+q-1, each
// run by A warps (A = the warps that hold the rows of the block still active at
// segment j; rows are ordered by non-increasing cut, so later segments need no
// more).  Warp w takes segment j + w / A and the rows (w mod A) * 32 + lane of
// the block; A * q <= 8.  Blocks whose long rows fill only a few warps (the rows
// nearest theta = 0) so pack several segments into one full CTA.
// cta_j packs j (bits 0-15), A - 1 (bits 16-19) and q - 1 (bits 20-23).
struct RecTask {
  int64_t rb, k;  // row block, half row of this thread
  int j;          // segment of this warp
  int jj, A, q;   // segment slot within the CTA, warps per segment, segments
  bool in;        // this warp has a segment
};
__device__ __forceinline__ RecTask rec_task(const RecArgs& R, int64_t cta) {
  const int code = R.cta_j[cta];
  RecTask t;
  t.A = ((code >> 16) & 15) + 1;
  t.q = ((code >> 20) & 15) + 1;
  const int w = threadIdx.x >> 5;
  t.jj = w / t.A;
  t.j = (code & 0xffff) + t.jj;
  t.in = t.jj < t.q;
  t.rb = R.cta_rb[cta];
  t.k = t.rb * RT + (w - t.jj * t.A) * 32 + (threadIdx.x & 31);
  return t;
}

// segments a row stores and runs: j0 .. nseg-1
__device__ __forceinline__ int nstored_of(const RecArgs& R, int64_t k) {
  return max(0, nseg_of(R, k) - R.j0);
}

// state (P, D) at n = n_lo of every row that runs segments past the head: the
// recurrence from n = 0 in the difference form, one thread per half row
__global__ void k_rec_lead(RecArgs R, double2* __restrict__ state) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R.H) return;
  if (nstored_of(R, k) == 0) return;
  const double xm1 = R.xm1[k];
  double P = 1.0, D = 1.0;
  for (int64_t n = 0; n < R.n_lo; ++n) {
    D = fma(R.ra[n] * xm1, P, R.rb[n] * D);
    P += D;
  }
  state[R.poff[k]] = make_double2(P, D);
}

// transfer matrix of one full segment: images of the basis states (1,0), (0,1)
__global__ void k_rec_basis(RecArgs R, double2* __restrict__ Tbuf) {
  const RecTask t = rec_task(R, blockIdx.x);
  const int64_t k = t.k;
  const int j = t.j;
  if (!t.in || k >= R.H) return;
  if (j >= nseg_of(R, k) - 1) return;
  const double xm1 = R.xm1[k];
  double P1 = 1.0, D1 = 0.0, P2 = 0.0, D2 = 1.0;
  const int64_t n0 = (int64_t)j * R.S;
  for (int64_t n = n0; n < n0 + R.S; ++n) {
    const double t = R.ra[n] * xm1;
    const double b = R.rb[n];
    D1 = fma(t, P1, b * D1);
    P1 += D1;
    D2 = fma(t, P2, b * D2);
    P2 += D2;
  }
  const int64_t o = 2 * (R.poff[k] + j - R.j0);
  Tbuf[o] = make_double2(P1, D1);
  Tbuf[o + 1] = make_double2(P2, D2);
}

__global__ void k_rec_scan(RecArgs R, const double2* __restrict__ Tbuf, double2* __restrict__ state) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= R.H) return;
  const int ns = nstored_of(R, k);
  if (ns == 0) return;
  const int64_t o = R.poff[k];
  double P = 1.0, D = 1.0;
  if (R.j0 > 0) {
    const double2 s0 = state[o];  // from k_rec_lead
    P = s0.x;
    D = s0.y;
  }
  state[o] = make_double2(P, D);
  for (int j = 0; j + 1 < ns; ++j) {
    const double2 a = Tbuf[2 * (o + j)], b = Tbuf[2 * (o + j) + 1];
    const double nP = a.x * P + b.x * D;
    const double nD = a.y * P + b.y * D;
    P = nP;
    D = nD;
    state[o + j + 1] = make_double2(P, D);
  }
}

// forward: the partial sums E (even n) and O (odd n) of half row k over segment
// j; false when the row's cut ends before the segment (o: its slot in the
// partial array).  rec_fwd_body takes the thread's (k, j) from CTA `cta` of the
// layout's CTA list.
template <typename T>
__device__ __forceinline__ bool rec_fwd_row(const RecArgs& R, int64_t k, int j, const T* __restrict__ c, int64_t& o,
                                            double2& EO) {
  const int cut = R.cut[k];
  if (j >= (cut + R.S - 1) / R.S) return false;
  o = R.poff[k] + j - R.j0;
  const double2 st = R.state[o];
  const double xm1 = R.xm1[k];
  double P = st.x, G = st.y / xm1;
  const int64_t n0 = (int64_t)j * R.S;
  const int64_t n1 = min(n0 + R.S, (int64_t)cut);
  double E = 0.0, O = 0.0;
  int64_t n = n0;
  for (; n + 1 < n1; n += 2) {
    E = fma((double)c[n], P, E);
    G = fma(R.ra[n], P, R.rb[n] * G);
    P = fma(xm1, G, P);
    O = fma((double)c[n + 1], P, O);
    G = fma(R.ra[n + 1], P, R.rb[n + 1] * G);
    P = fma(xm1, G, P);
  }
  if (n < n1) E = fma((double)c[n], P, E);
  EO = make_double2(E, O);
  return true;
}
template <typename T>
__device__ __forceinline__ bool rec_fwd_body(const RecArgs& R, int64_t cta, const T* __restrict__ c, int64_t& o,
                                             double2& EO) {
  const RecTask t = rec_task(R, cta);
  if (!t.in || t.k >= R.H) return false;
  return rec_fwd_row<T>(R, t.k, t.j, c, o, EO);
}

// FP32 form: the same segment sums with the recurrence in float-float and the
// products c_n P_n accumulated in Kahan-compensated float
__device__ __forceinline__ bool rec_fwd_row_ff(const RecArgs& R, int64_t k, int j, const float* __restrict__ c,
                                               int64_t& o, double2& EO) {
  const int cut = R.cut[k];
  if (j >= (cut + R.S - 1) / R.S) return false;
  o = R.poff[k] + j - R.j0;
  const double2 st = R.state[o];
  ffv P = ff_from(st.x), D = ff_from(st.y);
  const ffv xm1 = ff_from(R.xm1[k]);
  const int64_t n0 = (int64_t)j * R.S;
  const int64_t n1 = min(n0 + R.S, (int64_t)cut);
  float Es = 0.f, Ec = 0.f, Os = 0.f, Oc = 0.f;
  int64_t n = n0;
  for (; n + 1 < n1; n += 2) {
    kahan_add(Es, Ec, __fmul_rn(c[n], P.hi));
    D = ff_add(ff_mul_raw(ff_mul_raw(ff_ld(R.raf[n]), xm1), P), ff_mul_raw(ff_ld(R.rbf[n]), D));
    P = ff_add(P, D);
    kahan_add(Os, Oc, __fmul_rn(c[n + 1], P.hi));
    D = ff_add(ff_mul_raw(ff_mul_raw(ff_ld(R.raf[n + 1]), xm1), P), ff_mul_raw(ff_ld(R.rbf[n + 1]), D));
    P = ff_add(P, D);
  }
  if (n < n1) kahan_add(Es, Ec, __fmul_rn(c[n], P.hi));
  EO = make_double2((double)Es - (double)Ec, (double)Os - (double)Oc);
  return true;
}
__device__ __forceinline__ bool rec_fwd_body_ff(const RecArgs& R, int64_t cta, const float* __restrict__ c,
                                                int64_t& o, double2& EO) {
  const RecTask t = rec_task(R, cta);
  if (!t.in || t.k >= R.H) return false;
  return rec_fwd_row_ff(R, t.k, t.j, c, o, EO);
}

// The (half row, segment) of a thread of the packed forward launch (blockDim.x
// = 32 x warps per CTA): false when its lane has none
__device__ __forceinline__ bool fwd_pair(const RecArgs& R, int64_t& k, int& j) {
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw >= R.nfw) return false;
  const int code = R.fw_lane[gw * 32 + (threadIdx.x & 31)];
  if (code < 0) return false;
  k = (int64_t)R.fw_rb[gw] * RT + (code & 255);
  j = code >> 8;
  return k < R.H;
}

// The forward recurrence over the packed (row, segment) pairs: each thread the
// partial sums of one row over one segment (the same arithmetic, in the same
// order, as a thread of the per-segment CTAs of the layout's CTA list).
template <typename T>
__global__ void __launch_bounds__(RT) k_rec_fwd(RecArgs R, const T* __restrict__ c,
                                                double2* __restrict__ part) {
  c += (int64_t)blockIdx.y * R.N;
  part += (int64_t)blockIdx.y * R.nseg_total;
  int64_t k, o;
  int j;
  double2 EO;
  if (fwd_pair(R, k, j) && rec_fwd_row<T>(R, k, j, c, o, EO)) part[o] = EO;
}

__global__ void __launch_bounds__(RT) k_rec_fwd_ff(RecArgs R, const float* __restrict__ c,
                                                   double2* __restrict__ part) {
  c += (int64_t)blockIdx.y * R.N;
  part += (int64_t)blockIdx.y * R.nseg_total;
  int64_t k, o;
  int j;
  double2 EO;
  if (fwd_pair(R, k, j) && rec_fwd_row_ff(R, k, j, c, o, EO)) part[o] = EO;
}

// sum of a half row's segment partials; warp per row for rows [r0, r1) when
// warp_mode, thread per row otherwise
template <typename T>
__global__ void k_rec_fwd_reduce(RecArgs R, const double2* __restrict__ part, T* __restrict__ vrec,
                                 int64_t r0, int64_t r1, int warp_mode) {
  part += (int64_t)blockIdx.y * R.nseg_total;
  vrec += (int64_t)blockIdx.y * R.N;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double E = 0.0, O = 0.0;
  int64_t k;
  if (warp_mode) {
    k = r0 + gt / 32;
    const int lane = threadIdx.x & 31;
    if (k >= r1) return;  // whole warp leaves together
    const int ns = nstored_of(R, k);
    const int64_t o = R.poff[k];
    for (int j = lane; j < ns; j += 32) {
      const double2 p = part[o + j];
      E += p.x;
      O += p.y;
    }
    for (int off = 16; off > 0; off >>= 1) {
      E += __shfl_down_sync(0xffffffffu, E, off);
      O += __shfl_down_sync(0xffffffffu, O, off);
    }
    if (lane != 0) return;
  } else {
    k = r0 + gt;
    if (k >= r1) return;
    const int ns = nstored_of(R, k);
    const int64_t o = R.poff[k];
    for (int j = 0; j < ns; ++j) {
      const double2 p = part[o + j];
      E += p.x;
      O += p.y;
    }
  }
  vrec[k] = (T)(E + O);
  if (k != R.mid) vrec[R.N - 1 - k] = (T)(E - O);
}

// transposed: out_n = sum_k z_k P_n(x_k) over rows with n < cut(k).  A CTA takes
// 256 half rows x one segment of S columns.  Every 32 columns each lane
// writes its 32 values P_n(x_k) (0 past its cut) into its warp's tile; then lane
// i forms the dot product of tile column i with the warp's 32 row weights (a
// shared-memory transpose; the weight product rides in the fused multiply-add
// of the sum) into the warp's partial for that column.  Only warp-level
// synchronisation is needed until the end of the segment, where the 8 warp
// partials of each column are added into the row block's partial array.  Row
// weights: z_k + z_{N-1-k} for even n, z_k - z_{N-1-k} for odd n, by
// P_n(-x) = (-1)^n P_n(x); segments start at multiples of 32, so the parity of
// lane i's column is that of i.
constexpr int TP = 33;  // tile pitch

// The column partials of CTA `cta`: on return (after a CTA barrier) wsum[w][c]
// (sm + 8 * 32 * TP) holds warp w's sum of column c of its segment.
template <typename T>
__device__ __forceinline__ RecTask rec_t_body(const RecArgs& R, int64_t cta, const T* __restrict__ z, double* sm) {
  double* tile = sm;                  // [8][32][TP]
  double* wsum = sm + 8 * 32 * TP;    // [8][S] per-warp column partials
  double2* zt = reinterpret_cast<double2*>(wsum + 8 * R.S);  // [8][32] (z+, z-)
  const RecTask t = rec_task(R, cta);
  const int64_t rbk = t.rb;
  const int j = t.j;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = t.k;
  bool active = t.in && k < R.H;
  int cut = 0;
  double zp = 0.0, zm = 0.0, P = 0.0, G = 0.0, xm1 = 0.0;
  if (active) {
    cut = R.cut[k];
    active = j < (cut + R.S - 1) / R.S;
  }
  if (active) {
    double a = (double)z[k], b = (double)z[R.N - 1 - k];
    if (R.zw) {
      a *= R.zw[k];
      b *= R.zw[R.N - 1 - k];
    }
    zp = k == R.mid ? a : a + b;
    zm = k == R.mid ? a : a - b;
    const double2 st = R.state[R.poff[k] + j - R.j0];
    xm1 = R.xm1[k];
    P = st.x;
    G = st.y / xm1;
  } else {
    cut = 0;
  }
  zt[threadIdx.x] = make_double2(zp, zm);
  const int64_t n0s = (int64_t)j * R.S;
  const int64_t seg_end = min(n0s + R.S, (int64_t)R.maxcut[rbk]);
  double* mytile = tile + (w * 32 + lane) * TP;
  double* mysum = wsum + w * R.S;
  const double* zw = reinterpret_cast<const double*>(zt + w * 32) + (lane & 1);
  // columns past every cut of the warp's rows contribute nothing: the warp skips
  // them as a whole (a per-lane test would still issue the FP64 instructions)
  const int wcut = __reduce_max_sync(0xffffffffu, cut);
  for (int64_t n0 = n0s; n0 < seg_end; n0 += 32) {
    if (n0 >= wcut) {
      mysum[(n0 - n0s) + lane] = 0.0;
      continue;
    }
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      const int64_t n = n0 + i;
      double val = 0.0;
      if (n < cut) {
        val = P;
        G = fma(R.ra[n], P, R.rb[n] * G);
        P = fma(xm1, G, P);
      }
      mytile[i] = val;
    }
    __syncwarp();
    double colsum = 0.0;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) colsum = fma(zw[2 * r], tile[(w * 32 + r) * TP + lane], colsum);
    mysum[(n0 - n0s) + lane] = colsum;
    __syncwarp();
  }
  __syncthreads();
  return t;
}

template <typename T>
__global__ void __launch_bounds__(RT) k_rec_t(RecArgs R, const T* __restrict__ z,
                                              double* __restrict__ tbuf) {
  z += (int64_t)blockIdx.y * R.N;
  tbuf += (int64_t)blockIdx.y * R.tbuf_total;
  extern __shared__ double sm[];
  const RecTask t = rec_t_body<T>(R, blockIdx.x, z, sm);
  const double* wsum = sm + 8 * 32 * TP;
  const int64_t rbk = t.rb;
  // per segment of the CTA, the sum of its A warps' column partials
  const int jf = t.j - t.jj;
  for (int idx = threadIdx.x; idx < t.q * R.S; idx += RT) {
    const int sl = idx / R.S, c = idx - sl * R.S;
    const int64_t n0c = (int64_t)(jf + sl) * R.S;
    if (n0c + c >= (int64_t)R.maxcut[rbk]) continue;
    double s = 0.0;
    for (int a = 0; a < t.A; ++a) s += wsum[(sl * t.A + a) * R.S + c];
    tbuf[R.toff[rbk] + (n0c - R.n_lo) + c] = s;
  }
}

// FP32 form of k_rec_t: recurrence in float-float, products and the tile /
// warp sums in float, row-block partials stored in double.  On return (after a
// CTA barrier) wsum[w][c] (smf + 8 * 32 * TP) holds warp w's column sums.
__device__ __forceinline__ RecTask rec_t_body_ff(const RecArgs& R, int64_t cta, const float* __restrict__ z,
                                                 float* smf) {
  float* tile = smf;                 // [8][32][TP]
  float* wsum = smf + 8 * 32 * TP;   // [8][S]
  const RecTask t = rec_task(R, cta);
  const int64_t rbk = t.rb;
  const int j = t.j;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = t.k;
  bool active = t.in && k < R.H;
  int cut = 0;
  float zp = 0.f, zm = 0.f;
  ffv P = {0.f, 0.f}, D = {0.f, 0.f}, xm1 = {0.f, 0.f};
  if (active) {
    cut = R.cut[k];
    active = j < (cut + R.S - 1) / R.S;
  }
  if (active) {
    float a = z[k], b = z[R.N - 1 - k];
    if (R.zw) {
      a = (float)((double)a * R.zw[k]);
      b = (float)((double)b * R.zw[R.N - 1 - k]);
    }
    zp = k == R.mid ? a : a + b;
    zm = k == R.mid ? a : a - b;
    const double2 st = R.state[R.poff[k] + j - R.j0];
    P = ff_from(st.x);
    D = ff_from(st.y);
    xm1 = ff_from(R.xm1[k]);
  } else {
    cut = 0;
  }
  const int64_t n0s = (int64_t)j * R.S;
  const int64_t seg_end = min(n0s + R.S, (int64_t)R.maxcut[rbk]);
  float* mytile = tile + (w * 32 + lane) * TP;
  float* mysum = wsum + w * R.S;
  const int wcut = __reduce_max_sync(0xffffffffu, cut);
  for (int64_t n0 = n0s; n0 < seg_end; n0 += 32) {
    if (n0 >= wcut) {
      mysum[(n0 - n0s) + lane] = 0.f;
      continue;
    }
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
      const int64_t n = n0 + i;
      float val = 0.f;
      if (n < cut) {
        val = ((n & 1) ? zm : zp) * P.hi;
        D = ff_add(ff_mul_raw(ff_mul_raw(ff_ld(R.raf[n]), xm1), P), ff_mul_raw(ff_ld(R.rbf[n]), D));
        P = ff_add(P, D);
      }
      mytile[i] = val;
    }
    __syncwarp();
    float colsum = 0.f;
#pragma unroll 8
    for (int r = 0; r < 32; ++r) colsum += tile[(w * 32 + r) * TP + lane];
    mysum[(n0 - n0s) + lane] = colsum;
    __syncwarp();
  }
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(RT) k_rec_t_ff(RecArgs R, const float* __restrict__ z,
                                                 double* __restrict__ tbuf) {
  z += (int64_t)blockIdx.y * R.N;
  tbuf += (int64_t)blockIdx.y * R.tbuf_total;
  extern __shared__ float smf[];
  const RecTask t = rec_t_body_ff(R, blockIdx.x, z, smf);
  const float* wsum = smf + 8 * 32 * TP;
  const int64_t rbk = t.rb;
  const int jf = t.j - t.jj;
  for (int idx = threadIdx.x; idx < t.q * R.S; idx += RT) {
    const int sl = idx / R.S, c = idx - sl * R.S;
    const int64_t n0c = (int64_t)(jf + sl) * R.S;
    if (n0c + c >= (int64_t)R.maxcut[rbk]) continue;
    double s = 0.0;
    for (int a = 0; a < t.A; ++a) s += (double)wsum[(sl * t.A + a) * R.S + c];
    tbuf[R.toff[rbk] + (n0c - R.n_lo) + c] = s;
  }
}

// Transposed recurrence over packed (row, segment) pairs (fast layouts).  The
// pairs come ordered by segment, 32 to a warp, so a warp's lanes form runs of
// one segment each (several when a segment's active rows do not fill whole
// warps) and no lane idles where another segment has rows.  Per 32-column chunk
// (the same relative columns c0 .. c0 + 31 in every run) each lane writes its
// 32 values P_n(x_k) into its warp's tile; then lane i forms, per run, the dot
// product of tile column i over the run's rows with their weights and stores it
// in the run's slot.  Only warp-level synchronisation is used.  k_rec_tp_reduce
// adds a column's slots in slot order.  Row weights as in k_rec_t (z_k +
// z_{N-1-k} for even n, z_k - z_{N-1-k} for odd n: segments start at multiples
// of 32, so the parity of lane i's column is that of i).
struct TpLane {
  int64_t k;
  int j, slot, rc;  // segment, slot, columns of the segment below the row's cut
  bool active;
};
__device__ __forceinline__ TpLane tp_lane(const RecArgs& R, int64_t gw, int lane) {
  TpLane t;
  t.k = gw < R.ntw ? R.tw_k[gw * 32 + lane] : -1;
  t.slot = gw < R.ntw ? R.tw_slot[gw * 32 + lane] : -1;
  t.j = t.slot >= 0 ? R.tslot_j[t.slot] : 0;
  t.rc = 0;
  t.active = false;
  if (t.k >= 0 && t.k < R.H && t.slot >= 0) {
    const int cut = R.cut[t.k];
    if (t.j < (cut + R.S - 1) / R.S) {
      t.active = true;
      t.rc = min(cut - t.j * R.S, R.S);
    }
  }
  return t;
}

template <typename T>
__global__ void __launch_bounds__(RT) k_rec_tp(RecArgs R, const T* __restrict__ z, double* __restrict__ tpart) {
  z += (int64_t)blockIdx.y * R.N;
  tpart += (int64_t)blockIdx.y * R.tslots * R.S;
  extern __shared__ double sm[];
  const int wpc = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * wpc + w;
  if (gw >= R.ntw) return;  // whole warp: only warp-level synchronisation below
  double* tile = sm + w * 32 * TP;
  double2* zt = reinterpret_cast<double2*>(sm + wpc * 32 * TP) + w * 32;
  const TpLane t = tp_lane(R, gw, lane);
  double zp = 0.0, zm = 0.0, P = 0.0, G = 0.0, xm1 = 0.0;
  if (t.active) {
    double a = (double)z[t.k], b = (double)z[R.N - 1 - t.k];
    if (R.zw) {
      a *= R.zw[t.k];
      b *= R.zw[R.N - 1 - t.k];
    }
    zp = t.k == R.mid ? a : a + b;
    zm = t.k == R.mid ? a : a - b;
    const double2 st = R.state[R.poff[t.k] + t.j - R.j0];
    xm1 = R.xm1[t.k];
    P = st.x;
    G = st.y / xm1;
  }
  zt[lane] = make_double2(zp, zm);
  const unsigned full = 0xffffffffu;
  const int prev = __shfl_up_sync(full, t.slot, 1);
  const unsigned starts = __ballot_sync(full, lane == 0 || t.slot != prev);
  const int wrc = __reduce_max_sync(full, t.rc);
  const int64_t nb0 = (int64_t)t.j * R.S;
  const double* zw2 = reinterpret_cast<const double*>(zt) + (lane & 1);
  double* mytile = tile + lane * TP;
  __syncwarp();
  for (int c0 = 0; c0 < R.S; c0 += 32) {
    if (c0 < wrc) {
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        const int64_t n = nb0 + c0 + i;
        double val = 0.0;
        if (c0 + i < t.rc) {
          val = P;
          G = fma(R.ra[n], P, R.rb[n] * G);
          P = fma(xm1, G, P);
        }
        mytile[i] = val;
      }
      __syncwarp();
    }
    unsigned m = starts;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int e = m ? __ffs(m) - 1 : 32;
      const int sl = __shfl_sync(full, t.slot, b);
      double cs = 0.0;
      if (c0 < wrc)
        for (int r = b; r < e; ++r) cs = fma(zw2[2 * r], tile[r * TP + lane], cs);
      if (sl >= 0) tpart[(int64_t)sl * R.S + c0 + lane] = cs;
    }
    __syncwarp();
  }
}

// FP32 form of k_rec_tp: recurrence in float-float, products and the run sums in
// float, slots stored in double
__global__ void __launch_bounds__(RT) k_rec_tp_ff(RecArgs R, const float* __restrict__ z,
                                                  double* __restrict__ tpart) {
  z += (int64_t)blockIdx.y * R.N;
  tpart += (int64_t)blockIdx.y * R.tslots * R.S;
  extern __shared__ float smf[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;
  if (gw >= R.ntw) return;
  float* tile = smf + w * 32 * TP;
  const TpLane t = tp_lane(R, gw, lane);
  float zp = 0.f, zm = 0.f;
  ffv P = {0.f, 0.f}, D = {0.f, 0.f}, xm1 = {0.f, 0.f};
  if (t.active) {
    float a = z[t.k], b = z[R.N - 1 - t.k];
    if (R.zw) {
      a = (float)((double)a * R.zw[t.k]);
      b = (float)((double)b * R.zw[R.N - 1 - t.k]);
    }
    zp = t.k == R.mid ? a : a + b;
    zm = t.k == R.mid ? a : a - b;
    const double2 st = R.state[R.poff[t.k] + t.j - R.j0];
    P = ff_from(st.x);
    D = ff_from(st.y);
    xm1 = ff_from(R.xm1[t.k]);
  }
  const unsigned full = 0xffffffffu;
  const int prev = __shfl_up_sync(full, t.slot, 1);
  const unsigned starts = __ballot_sync(full, lane == 0 || t.slot != prev);
  const int wrc = __reduce_max_sync(full, t.rc);
  const int64_t nb0 = (int64_t)t.j * R.S;
  float* mytile = tile + lane * TP;
  for (int c0 = 0; c0 < R.S; c0 += 32) {
    if (c0 < wrc) {
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        const int64_t n = nb0 + c0 + i;
        float val = 0.f;
        if (c0 + i < t.rc) {
          val = ((i & 1) ? zm : zp) * P.hi;
          D = ff_add(ff_mul_raw(ff_mul_raw(ff_ld(R.raf[n]), xm1), P), ff_mul_raw(ff_ld(R.rbf[n]), D));
          P = ff_add(P, D);
        }
        mytile[i] = val;
      }
      __syncwarp();
    }
    unsigned m = starts;
    while (m) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const int e = m ? __ffs(m) - 1 : 32;
      const int sl = __shfl_sync(full, t.slot, b);
      float cs = 0.f;
      if (c0 < wrc)
        for (int r = b; r < e; ++r) cs += tile[r * TP + lane];
      if (sl >= 0) tpart[(int64_t)sl * R.S + c0 + lane] = (double)cs;
    }
    __syncwarp();
  }
}

// out_n = the sum of segment j = n / S's slots at column n - j S, in slot order
// (columns below n_lo belong to the dense head block and get 0 here), times n +
// 1/2 when the chain scales its output
template <typename T>
__global__ void k_rec_tp_reduce(RecArgs R, const double* __restrict__ tpart, T* __restrict__ out) {
  const int64_t bt = blockIdx.y;
  tpart += bt * R.tslots * R.S;
  out += bt * R.N;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= R.N) return;
  double s = 0.0;
  if (n >= R.n_lo) {
    const int64_t jj = n / R.S - R.j0;
    if (jj < R.tsegs) {
      const int64_t c = n - (n / R.S) * R.S;
      for (int64_t sl = R.tseg_begin[jj]; sl < R.tseg_begin[jj + 1]; ++sl) s += tpart[sl * R.S + c];
    }
  }
  if (R.scale_out) s *= (double)n + 0.5;
  out[n] = (T)s;
}

// Column sums of the row blocks' partials: out_n = sum over row blocks with
// cut > n of tbuf[toff[rb] + n - n_lo] (row blocks come in order of non-increasing
// cut, so the contributing blocks are a prefix; columns below n_lo belong to the
// dense head block and get 0 here).  Columns [n_lo, n_heavy) lie below the
// cuts of more than 32 blocks: k_rec_t_reduce_part sums them in chunks of 64
// row blocks (grid: column groups x chunks, one round of independent loads per
// warp) into a small scratch; k_rec_t_reduce_final adds the chunk sums of those
// columns and sums the other columns' few blocks directly, one thread per column.
constexpr int RB_CHUNK = 64;

__global__ void k_rec_t_reduce_part(RecArgs R, const double* __restrict__ tbuf) {
  __shared__ double red[8][32];
  const int64_t bt = blockIdx.z;
  tbuf += bt * R.tbuf_total;
  double* scr = R.rscratch + bt * R.rchunks * R.n_heavy;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = R.n_lo + (int64_t)blockIdx.x * 32 + lane;
  const int64_t rbc = (int64_t)blockIdx.y * RB_CHUNK;
  double s = 0.0;
  if (n < R.n_heavy) {
    double v[RB_CHUNK / 8];
#pragma unroll
    for (int u = 0; u < RB_CHUNK / 8; ++u) {
      const int64_t rb = rbc + w + 8 * u;
      v[u] = (rb < R.nblocks && (int64_t)R.maxcut[rb] > n) ? tbuf[R.toff[rb] + n - R.n_lo] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < RB_CHUNK / 8; ++u) s += v[u];
  }
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && n < R.n_heavy) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    scr[blockIdx.y * R.n_heavy + n] = t;
  }
}

template <typename T>
__global__ void k_rec_t_reduce_final(RecArgs R, const double* __restrict__ tbuf, T* __restrict__ out) {
  const int64_t bt = blockIdx.y;
  tbuf += bt * R.tbuf_total;
  out += bt * R.N;
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= R.N) return;
  double s = 0.0;
  if (n < R.n_lo) {
    // the dense head block's columns: no recurrence contributions
  } else if (n < R.n_heavy) {
    const double* scr = R.rscratch + bt * R.rchunks * R.n_heavy + n;
    for (int64_t c = 0; c < R.rchunks; ++c) s += scr[c * R.n_heavy];
  } else {
    constexpr int U = 4;
    for (int64_t rb0 = 0; rb0 < R.nblocks; rb0 += U) {
      double v[U];
      bool more = true;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t rb = rb0 + u;
        const bool in = rb < R.nblocks && (int64_t)R.maxcut[rb] > n;
        v[u] = in ? tbuf[R.toff[rb] + n - R.n_lo] : 0.0;
        if (u == U - 1) more = in;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) s += v[u];
      if (!more) break;
    }
  }
  if (R.scale_out) s *= (double)n + 0.5;
  out[n] = (T)s;
}

// Direct method over many small transforms in one launch: each job is one
// transform whose direct layout is a single CTA (one row block, one segment per
// row: N <= S), so the CTA finishes the whole transform, reductions included.
// A persistent grid strides over the job table fixed at batch creation.  The
// arithmetic is that of the per-plan chain step for step (partial sums added
// from 0.0 in the same order, the same casts), so the outputs are bitwise those
// of single-plan calls.
struct DirectJob {
  int32_t arg;  // index of the transform's RecArgs
  int32_t pad;
  const void* in;
  void* out;
};

template <typename T>
__global__ void __launch_bounds__(RT) k_direct_fwd_multi(const RecArgs* __restrict__ args,
                                                         const DirectJob* __restrict__ jobs, int64_t njobs) {
  for (int64_t jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
    const DirectJob J = jobs[jb];
    const RecArgs& R = args[J.arg];
    int64_t o;
    double2 EO;
    bool have;
    if constexpr (sizeof(T) == 4)
      have = rec_fwd_body_ff(R, 0, (const float*)J.in, o, EO);
    else
      have = rec_fwd_body<T>(R, 0, (const T*)J.in, o, EO);
    const RecTask t = rec_task(R, 0);
    if (t.in && t.k < R.H) {
      // the row's one partial, added from 0.0 as the row reduction does
      const double E = 0.0 + (have ? EO.x : 0.0), O = 0.0 + (have ? EO.y : 0.0);
      T* f = (T*)J.out;
      f[t.k] = (T)(E + O);
      if (t.k != R.mid) f[R.N - 1 - t.k] = (T)(E - O);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) k_direct_t_multi(const RecArgs* __restrict__ args,
                                                       const DirectJob* __restrict__ jobs, int64_t njobs) {
  extern __shared__ double sm[];
  for (int64_t jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
    const DirectJob J = jobs[jb];
    const RecArgs& R = args[J.arg];
    RecTask t;
    if constexpr (sizeof(T) == 4)
      t = rec_t_body_ff(R, 0, (const float*)J.in, reinterpret_cast<float*>(sm));
    else
      t = rec_t_body<T>(R, 0, (const T*)J.in, sm);
    const int64_t mc = R.maxcut[0];
    T* out = (T*)J.out;
    for (int c = threadIdx.x; c < R.N; c += RT) {
      // the block partial (warp partials from 0.0), then the column reduction
      // over the one row block (from 0.0) and the output scale
      double s = 0.0;
      if (c < mc) {
        if constexpr (sizeof(T) == 4) {
          const float* wsum = reinterpret_cast<const float*>(sm) + 8 * 32 * TP;
          for (int a = 0; a < t.A; ++a) s += (double)wsum[a * R.S + c];
        } else {
          const double* wsum = sm + 8 * 32 * TP;
          for (int a = 0; a < t.A; ++a) s += wsum[a * R.S + c];
        }
      }
      double v = 0.0 + s;
      if (R.scale_out) v *= (double)c + 0.5;
      out[c] = (T)v;
    }
    __syncthreads();  // the next job rewrites the tiles and partials
  }
}

}  // namespace

int launch_rec_xm1(Plan& P, RecLayout& L, int legendre) {
  if (L.H == 0) return GBDLT_OK;
  k_rec_xm1<<<(unsigned)((L.H + 255) / 256), 256, 0, P.stream>>>(L.xm1, legendre ? P.theta : nullptr, L.H, P.p.N);
  count_launch();
  return check_launch();
}

int launch_rec_state_init(Plan& P, RecLayout& L) {
  if (L.H == 0 || L.nseg_total == 0) return GBDLT_OK;
  double2* Tbuf = nullptr;
  if (dev_malloc((void**)&Tbuf, sizeof(double2) * 2 * (size_t)L.nseg_total) != cudaSuccess) {
    cudaGetLastError();
    return GBDLT_ERR_OOM;
  }
  RecArgs R = rec_args(P, L);
  if (L.j0 > 0) {
    k_rec_lead<<<(unsigned)((L.H + 127) / 128), 128, 0, P.stream>>>(R, L.state);
    count_launch();
  }
  if (L.ncta > 0) {
    k_rec_basis<<<(unsigned)L.ncta, RT, 0, P.stream>>>(R, Tbuf);
    count_launch();
  }
  k_rec_scan<<<(unsigned)((L.H + 127) / 128), 128, 0, P.stream>>>(R, Tbuf, L.state);
  count_launch();
  int st = check_launch();
  cudaStreamSynchronize(P.stream);
  cudaFree(Tbuf);
  return st;
}

template <typename T>
int launch_rec_forward(Plan& P, RecLayout& L, const T* c, T* vrec, int64_t nb) {
  RecArgs R = rec_args(P, L);
  if (L.H == 0) return GBDLT_OK;
  // (no segments at all when the head block and the bands cover every column)
  if (L.nfw > 0) {
    const dim3 grid((unsigned)((L.nfw + L.fwpc - 1) / L.fwpc), (unsigned)nb);
    if constexpr (sizeof(T) == 4) {
      k_rec_fwd_ff<<<grid, 32 * L.fwpc, 0, P.stream>>>(R, (const float*)c, L.part);
    } else {
      k_rec_fwd<T><<<grid, 32 * L.fwpc, 0, P.stream>>>(R, c, L.part);
    }
    launched(P, "rec_fwd", (double)nb * 7.0 * (double)L.half_steps,
             (double)nb * ((double)sizeof(T) * P.p.N + 32.0 * (double)L.nseg_total));
  }
  if (L.n_long > 0) {
    const int64_t threads = L.n_long * 32;
    k_rec_fwd_reduce<T><<<dim3((unsigned)((threads + 255) / 256), (unsigned)nb), 256, 0, P.stream>>>(
        R, L.part, vrec, 0, L.n_long, 1);
    launched(P, "rec_fwd_reduce", 0.0, 0.0);
  }
  if (L.H > L.n_long) {
    const int64_t rows = L.H - L.n_long;
    k_rec_fwd_reduce<T><<<dim3((unsigned)((rows + 255) / 256), (unsigned)nb), 256, 0, P.stream>>>(
        R, L.part, vrec, L.n_long, L.H, 0);
    launched(P, "rec_fwd_reduce", (double)nb * 2.0 * (double)L.nseg_total,
             (double)nb * (16.0 * (double)L.nseg_total + (double)sizeof(T) * P.p.N));
  }
  return check_launch();
}

template <typename T>
int launch_rec_transpose(Plan& P, RecLayout& L, const T* z, T* out, int64_t nb, const double* zw,
                         int scale_out) {
  RecArgs R = rec_args(P, L);
  R.zw = zw;
  R.scale_out = scale_out;
  if (L.H == 0) return GBDLT_OK;
  if (L.ntw > 0) {
    // fast layouts: the packed launch and its slot reduction
    const size_t smem_tp = (size_t)L.twpc * 32 * (sizeof(T) * TP + (sizeof(T) == 8 ? 16 : 0));
    static bool attr_tp = false;
    const dim3 grid((unsigned)((L.ntw + L.twpc - 1) / L.twpc), (unsigned)nb);
    if constexpr (sizeof(T) == 4) {
      if (!attr_tp) {
        cudaFuncSetAttribute(k_rec_tp_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * 32 * 4 * TP));
        attr_tp = true;
      }
      k_rec_tp_ff<<<grid, 32 * L.twpc, smem_tp, P.stream>>>(R, (const float*)z, L.tpart);
    } else {
      if (!attr_tp) {
        cudaFuncSetAttribute(k_rec_tp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(8 * 32 * (8 * TP + 16)));
        attr_tp = true;
      }
      k_rec_tp<T><<<grid, 32 * L.twpc, smem_tp, P.stream>>>(R, z, L.tpart);
    }
    launched(P, "rec_t", (double)nb * 7.0 * (double)L.half_steps,
             (double)nb * ((double)sizeof(T) * P.p.N + 16.0 * (double)L.nseg_total +
                           8.0 * (double)L.tslots * L.S));
    k_rec_tp_reduce<T><<<dim3((unsigned)((P.p.N + 255) / 256), (unsigned)nb), 256, 0, P.stream>>>(R, L.tpart, out);
    launched(P, "rec_t_reduce", (double)nb * (double)L.tslots * L.S,
             (double)nb * (8.0 * (double)L.tslots * L.S + (double)sizeof(T) * P.p.N));
    return check_launch();
  }
  const size_t smem = sizeof(T) * (8 * 32 * TP + 8 * (size_t)L.S) + (sizeof(T) == 8 ? 16 * RT : 0);
  static bool attr_set = false;
  if (L.ncta > 0) {
    if constexpr (sizeof(T) == 4) {
      if (!attr_set) {
        cudaFuncSetAttribute(k_rec_t_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
      }
      k_rec_t_ff<<<dim3((unsigned)L.ncta, (unsigned)nb), RT, smem, P.stream>>>(R, (const float*)z, L.tbuf);
    } else {
      if (!attr_set) {
        cudaFuncSetAttribute(k_rec_t<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = true;
      }
      k_rec_t<T><<<dim3((unsigned)L.ncta, (unsigned)nb), RT, smem, P.stream>>>(R, z, L.tbuf);
    }
    launched(P, "rec_t", (double)nb * 7.0 * (double)L.half_steps,
             (double)nb * ((double)sizeof(T) * P.p.N + 16.0 * (double)L.nseg_total + 8.0 * (double)L.tbuf_total));
  }
  if (R.n_heavy > R.n_lo) {
    k_rec_t_reduce_part<<<dim3((unsigned)((R.n_heavy - R.n_lo + 31) / 32), (unsigned)R.rchunks, (unsigned)nb), 256,
                          0, P.stream>>>(R, L.tbuf);
    count_launch();
  }
  k_rec_t_reduce_final<T><<<dim3((unsigned)((P.p.N + 255) / 256), (unsigned)nb), 256, 0, P.stream>>>(R, L.tbuf,
                                                                                                   out);
  launched(P, "rec_t_reduce", (double)nb * (double)L.tbuf_total,
           (double)nb * (8.0 * (double)L.tbuf_total + (double)sizeof(T) * P.p.N));
  return check_launch();
}

struct DirectMulti {
  int prec = GBDLT_FP64;
  int dir = 0;
  int64_t njobs = 0;
  RecArgs* args = nullptr;  // device [groups]
  DirectJob* jobs = nullptr;
  unsigned grid = 0;
  size_t smem = 0;
};

bool direct_fusable(const Plan& P) {
  const RecLayout& L = P.drec;
  return P.has_direct && P.p.N > 1 && L.H > 0 && L.ncta == 1 && L.nblocks == 1 && L.j0 == 0 &&
         L.nseg_total == L.H && L.n_heavy <= 0 && P.p.N <= L.S;
}

int direct_multi_create(const std::vector<DirectGroupRef>& groups, int prec, int dir, DirectMulti** out) {
  *out = nullptr;
  if (groups.empty()) return GBDLT_OK;
  DirectMulti* d = new (std::nothrow) DirectMulti();
  if (!d) return GBDLT_ERR_OOM;
  d->prec = prec;
  d->dir = dir;
  const size_t es = prec == GBDLT_FP64 ? 8 : 4;
  std::vector<RecArgs> args;
  std::vector<std::pair<int64_t, DirectJob>> jobs;  // (N, job), longest first
  for (const DirectGroupRef& g : groups) {
    if (!direct_fusable(*g.plan)) {
      direct_multi_free(d);
      return GBDLT_ERR_INVALID_ARG;
    }
    RecArgs R = rec_args(*g.plan, g.plan->drec);
    if (dir == 1) {
      R.zw = g.plan->w;
      R.scale_out = 1;
    }
    const int64_t N = g.plan->p.N;
    for (int64_t i = 0; i < g.count; ++i) {
      DirectJob J;
      J.arg = (int32_t)args.size();
      J.pad = 0;
      J.in = (const char*)g.in + (size_t)(i * N) * es;
      J.out = (char*)g.out + (size_t)(i * N) * es;
      jobs.push_back({N, J});
    }
    args.push_back(R);
  }
  std::stable_sort(jobs.begin(), jobs.end(),
                   [](const std::pair<int64_t, DirectJob>& a, const std::pair<int64_t, DirectJob>& b) {
                     return a.first > b.first;
                   });
  std::vector<DirectJob> table;
  for (auto& j : jobs) table.push_back(j.second);
  d->njobs = (int64_t)table.size();
  if (dev_malloc((void**)&d->args, sizeof(RecArgs) * args.size()) != cudaSuccess ||
      dev_malloc((void**)&d->jobs, sizeof(DirectJob) * table.size()) != cudaSuccess) {
    cudaGetLastError();
    direct_multi_free(d);
    return GBDLT_ERR_OOM;
  }
  if (cudaMemcpy(d->args, args.data(), sizeof(RecArgs) * args.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d->jobs, table.data(), sizeof(DirectJob) * table.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    direct_multi_free(d);
    return GBDLT_ERR_CUDA;
  }
  // persistent grid: the CTAs the SMs hold at once, or one per job
  const void* fn = nullptr;
  int S = 0;
  for (const DirectGroupRef& g : groups) S = std::max(S, g.plan->drec.S);
  if (dir == 0) {
    fn = prec == GBDLT_FP64 ? (const void*)k_direct_fwd_multi<double> : (const void*)k_direct_fwd_multi<float>;
  } else {
    d->smem = es * (8 * 32 * TP + 8 * (size_t)S) + (es == 8 ? 16 * RT : 0);
    fn = prec == GBDLT_FP64 ? (const void*)k_direct_t_multi<double> : (const void*)k_direct_t_multi<float>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d->smem) != cudaSuccess) {
      direct_multi_free(d);
      return GBDLT_ERR_CUDA;
    }
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RT, d->smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    sms = 1;
  }
  d->grid = (unsigned)std::min<int64_t>(d->njobs, (int64_t)per_sm * sms);
  *out = d;
  return GBDLT_OK;
}

int direct_multi_launch(DirectMulti* d, cudaStream_t s) {
  if (!d || d->njobs == 0) return GBDLT_OK;
  if (d->dir == 0) {
    if (d->prec == GBDLT_FP64)
      k_direct_fwd_multi<double><<<d->grid, RT, 0, s>>>(d->args, d->jobs, d->njobs);
    else
      k_direct_fwd_multi<float><<<d->grid, RT, 0, s>>>(d->args, d->jobs, d->njobs);
  } else {
    if (d->prec == GBDLT_FP64)
      k_direct_t_multi<double><<<d->grid, RT, d->smem, s>>>(d->args, d->jobs, d->njobs);
    else
      k_direct_t_multi<float><<<d->grid, RT, d->smem, s>>>(d->args, d->jobs, d->njobs);
  }
  count_launch();
  return check_launch();
}

int64_t direct_multi_jobs(const DirectMulti* d) { return d ? d->njobs : 0; }

void direct_multi_free(DirectMulti* d) {
  if (!d) return;
  if (d->args) cudaFree(d->args);
  if (d->jobs) cudaFree(d->jobs);
  delete d;
}

template int launch_rec_forward<double>(Plan&, RecLayout&, const double*, double*, int64_t);
template int launch_rec_forward<float>(Plan&, RecLayout&, const float*, float*, int64_t);
template int launch_rec_transpose<double>(Plan&, RecLayout&, const double*, double*, int64_t, const double*, int);
template int launch_rec_transpose<float>(Plan&, RecLayout&, const float*, float*, int64_t, const double*, int);

}  // namespace gbdlt
