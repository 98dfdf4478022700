// Gauss-Legendre nodes and weights on the GPU (Sec. 2.1-2.2).
//
// One thread per node k < ceil(N/2) (theta < pi/2); the other half follows from
// the symmetry theta_{N-1-k} = pi - theta_k, w_{N-1-k} = w_k.  Newton's method
// runs in delta = theta - theta*_k around the cheb* point
// theta*_k = (k+3/4)pi/(N+1/2) of Sec. 2.2, which Lemma 2.3 places within
// 1/(3 pi (2N+1)) of the root (interior nodes start from the first-order
// correction of that point, see k_legpts).  Working in delta keeps the phase of P_N exact:
// (N+1/2) theta*_k - pi/4 = (k+1/2) pi, so cos/sin of the phase are those of the
// small angle eps = (N+1/2) delta, with no large-argument reduction.
//
// P_N(cos theta) and dP_N/dtheta are evaluated by one of three methods:
//  * N <= 64: the three-term recurrence in difference form,
//      D_{n+1} = [(2n+1)(x-1) P_n + n D_n]/(n+1),  P_{n+1} = P_n + D_{n+1},
//    with x - 1 = -2 sin^2(theta/2) (no cancellation near x = 1);
//  * N sin(theta) >= 25: the large-degree asymptotic expansion whose leading
//    term is quoted in Sec. 2.2 (Stieltjes), carried to the order where the
//    next term is below 1e-18 of the leading amplitude:
//      P_N(cos t) = C_N sum_m h_{m,N} cos((N+m+1/2)t - (m+1/2)pi/2) / (2 sin t)^{m+1/2},
//      C_N = sqrt(4/pi) Gamma(N+1)/Gamma(N+3/2),
//      h_{0,N} = 1, h_{m+1,N} = h_{m,N} (m+1/2)^2 / ((m+1)(N+m+3/2));
//  * otherwise (the 8 nodes nearest theta = 0): the terminating hypergeometric
//    series P_N(cos t) = sum_j (-N)_j (N+1)_j / (j!)^2 s^j, s = sin^2(t/2),
//    summed in double-double (its terms reach ~1e10 before they cancel) by one
//    warp per node (end_node, the first blocks of k_legpts): lane l holds terms 3l..3l+2, obtains the
//    first of them as a prefix product of the term ratios over the lanes below,
//    and the sums are reduced across the warp.  These nodes start Newton from
//    j_{0,k+1}/(N+1/2), the zeros of Hilb's Bessel approximation
//    P_N(cos t) ~ sqrt(t / sin t) J_0((N+1/2) t).
// Weight: w_k = 2 / (dP_N/dtheta)^2 at the root (Gauss-Legendre weight written
// in theta).  Outputs per node: theta_k, x_k = cos theta_k, w_k and
// t_k = N * (theta_k - (k+1/2)pi/N), the scaled offset from the cheb1 grid used
// by the Taylor series of Sec. 2.1 (computed from the exact difference
// theta*_k - theta^cheb1_k = pi (N-2k-1) / (4N(N+1/2)) plus delta, so it keeps
// full relative accuracy).
#include <algorithm>
#include <cmath>

#include "gbdlt_internal.cuh"

namespace gbdlt {

namespace {

constexpr double kPi = 3.141592653589793238;

struct PD {
  double p, dp;
  double cot;  // cot(theta) at the evaluation point
};

// h_{m,N} of the expansion for m < kMaxTerms; the same for every node of a plan,
// so the host computes them once per launch
constexpr int kMaxTerms = 40;
struct HTab {
  double h[kMaxTerms];
};

__device__ PD eval_rec(int64_t N, double s, double c, double sh) {
  // s = sin(theta), c = cos(theta), sh = sin(theta/2)
  double xm1 = -2.0 * sh * sh;
  double P = 1.0, D = 1.0;
  for (int64_t n = 0; n < N; ++n) {
    double Dn = ((double)(2 * n + 1) * xm1 * P + (double)n * D) / (double)(n + 1);
    P += Dn;
    D = Dn;
  }
  // P_{N-1} - x P_N = -(x-1) P_N - D_N
  PD r;
  r.p = P;
  r.dp = (double)N * (xm1 * P + D) / s;
  r.cot = c / s;
  return r;
}

// Nh = N + 1/2
__device__ PD eval_asy(double Nh, int64_t k, double d, double s, double c, double CN, const HTab& H) {
  const double eps = Nh * d;
  const double e2 = eps * eps;
  // sin/cos of |eps| <= 0.06 by Taylor polynomials (error < 1e-19)
  double se = eps * (1.0 + e2 * (-1.0 / 6 + e2 * (1.0 / 120 + e2 * (-1.0 / 5040 + e2 * (1.0 / 362880)))));
  double ce = 1.0 + e2 * (-0.5 + e2 * (1.0 / 24 + e2 * (-1.0 / 720 + e2 * (1.0 / 40320))));
  const double sg = (k & 1) ? -1.0 : 1.0;
  double cr = -sg * se, ci = sg * ce;  // e^{i phi_0}, phi_0 = (k+1/2)pi + eps
  const double rr = s, ri = -c;        // e^{i(theta - pi/2)}
  // (2 sin theta)^{-1/2} by one reciprocal square root; g = 1/(2 sin theta) and
  // 1/sin theta follow from it by products
  const double sg0 = rsqrt(2.0 * s);
  const double g = sg0 * sg0;
  const double inv_s = 2.0 * g;
  const double cot = c * inv_s;
  double gm = sg0;  // g^{m+1/2}
  double P = 0.0, dP = 0.0;
  double mh = 0.5, nmh = Nh;  // m + 1/2 and N + m + 1/2, exact
  for (int m = 0; m < kMaxTerms - 1; ++m) {
    const double term = H.h[m] * gm;
    P += term * cr;
    dP += term * (-nmh * ci - mh * cot * cr);
    mh += 1.0;
    nmh += 1.0;
    gm *= g;
    const double ncr = cr * rr - ci * ri;
    ci = cr * ri + ci * rr;
    cr = ncr;
    if (H.h[m + 1] * gm < 1e-18 * sg0) break;
  }
  PD r;
  r.p = CN * P;
  r.dp = CN * dP;
  r.cot = cot;
  return r;
}

// Per-plan constants of the node kernels (host-computed): 1/(N+1/2) and the
// first-order start factor 1/(8 (N+1/2)(N+3/2)).
struct NodeConst {
  double inv_Nh;
  double c1;
};

// node k >= kend (k < kend: end_node)
__device__ __forceinline__ void interior_node(int64_t N, int64_t k, double CN, const HTab& H, const NodeConst& K,
                                              double* __restrict__ theta, double* __restrict__ x,
                                              double* __restrict__ w, double* __restrict__ tN,
                                              int* __restrict__ status, int max_iter) {
  const double Nh = (double)N + 0.5;
  const double inv_Nh = K.inv_Nh;
  const double th0 = ((double)k + 0.75) * kPi * inv_Nh;
  double s0, c0;
  sincospi(((double)k + 0.75) * inv_Nh, &s0, &c0);
  const int mode = N <= 64 ? 0 : 1;
  // interior nodes start from the zero of the first two terms of the expansion:
  // cos(phi_0) + h_1 cos(phi_1) / (2 sin theta) = 0 gives, to first order,
  // (N+1/2) delta = cot(theta) / (8 (N+3/2)), i.e. about 1000 times closer than theta*.
  // A start needs no more than float accuracy in cot (its error 1e-7 of a
  // correction of 1e-13 or less): 1/sin theta by the float reciprocal
  // (sin theta* >= 25/N >= 1.5e-6 here, well inside float range).
  double d = mode == 1 ? c0 * (double)__frcp_rn((float)s0) * K.c1 : 0.0;
  bool ok = false;
  PD r;
  double s = s0, c = c0, sh = 0, ch = 0, dp_final = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    // sin/cos of theta = th0 + d by the angle-addition formula; |d| <= 1/(3 pi (2N+1))
    // (Lemma 2.3), so the Taylor polynomials below are exact to < 1e-20
    const double d2 = d * d;
    const double sd = d * (1.0 - d2 * (1.0 / 6.0) *
                                     (1.0 - d2 * (1.0 / 20.0) * (1.0 - d2 * (1.0 / 42.0) * (1.0 - d2 * (1.0 / 72.0)))));
    const double cd =
        1.0 - d2 * 0.5 *
                  (1.0 - d2 * (1.0 / 12.0) *
                             (1.0 - d2 * (1.0 / 30.0) * (1.0 - d2 * (1.0 / 56.0) * (1.0 - d2 * (1.0 / 90.0)))));
    s = s0 * cd + c0 * sd;
    c = c0 * cd - s0 * sd;
    if (mode == 0) {
      double th = th0 + d;
      sincos(0.5 * th, &sh, &ch);
      r = eval_rec(N, s, c, sh);
    } else {
      r = eval_asy(Nh, k, d, s, c, CN, H);
    }
    const double step = r.p / r.dp;
    d -= step;
    if (!(fabs(d) < 1.0)) break;  // diverged (NaN or runaway)
    // Newton's error after this step is about (f''/2f') step^2 = (cot(theta)/2) step^2
    // (at a root Legendre's equation gives P'' = -cot(theta) P').  Stop once that
    // is far below the rounding floor of the evaluation (~u/N in theta) and the
    // step is small enough for the one-step derivative update below to keep the
    // weight to ~1e-17 relative ((step N)^2 / 2).
    const double a_step = fabs(step);
    if (a_step * (double)N <= 1e-8 && (0.5 * fabs(r.cot) + 1.0) * a_step * a_step * (double)N <= 1e-18) {
      // dP/dtheta at the updated point by one Taylor step, with the second
      // derivative from Legendre's equation in theta:
      //   P'' = -cot(theta) P' - N(N+1) P   (step^2 N^3 is below 1e-20 here)
      dp_final = r.dp + step * (r.cot * r.dp + (double)N * ((double)N + 1.0) * r.p);
      // cos/sin at the updated point (theta decreased by step)
      const double cn = c + s * step;
      s = s - c * step;
      c = cn;
      ok = true;
      break;
    }
  }
  if (!ok) atomicOr(status, 1);
  const double th = th0 + d;
  const double wk = 2.0 / (dp_final * dp_final);
  const double xk = c;
  const double tk = kPi * (double)(N - 2 * k - 1) * (0.25 * inv_Nh) + (double)N * d;
  theta[k] = th;
  x[k] = xk;
  w[k] = wk;
  tN[k] = tk;
  const int64_t km = N - 1 - k;
  if (km != k) {
    theta[km] = kPi - th;
    x[km] = -xk;
    w[km] = wk;
    tN[km] = -tk;
  }
}

// zeros j_{0,m}, m = 1..10, of the Bessel function J_0 (DLMF 10.21)
__constant__ double kJ0Zeros[10] = {2.404825557695772768622, 5.520078110286310649597, 8.653727912911012216954,
                                    11.79153443901428161374, 14.93091770848778594776, 18.07106396791092254315,
                                    21.21163662987925895908, 24.35247153074930273706, 27.49347913204025479588,
                                    30.63460646843197511755};
constexpr int kMaxEnds = 10;

__device__ __forceinline__ ddv shfl_up_dd(ddv v, int off) {
  return {__shfl_up_sync(0xffffffffu, v.hi, off), __shfl_up_sync(0xffffffffu, v.lo, off)};
}
__device__ __forceinline__ ddv shfl_xor_dd(ddv v, int m) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// P_N(cos t) and dP_N/dt from the hypergeometric series by one warp (every lane
// returns lane 0's values).  Term ratio t_{j+1}/t_j = -(N-j)(N+j+1)/(j+1)^2 s;
// with N sin t < 25 the terms fall below 1e-90 of the largest before j = 96.
__device__ PD eval_series_warp(int64_t N, double sh, double ch, int lane) {
  const double sq = sh * sh;  // s = sin^2(t/2)
  const double Nd = (double)N;
  ddv rho[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int j = 3 * lane + q;
    if ((int64_t)j < N) {
      const double num = -(Nd - j) * (Nd + j + 1.0);  // exact in double for N <= 2^26
      const double den = (double)(j + 1) * (double)(j + 1);
      rho[q] = dd_mul_d(dd_div_dd(num, den), sq);
    } else {
      rho[q] = {0.0, 0.0};  // (-N)_j = 0 for j > N
    }
  }
  // inclusive prefix product of the lanes' ratio products, then the exclusive one
  ddv R = dd_mul(dd_mul(rho[0], rho[1]), rho[2]);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const ddv v = shfl_up_dd(R, off);
    if (lane >= off) R = dd_mul(v, R);
  }
  ddv t0 = shfl_up_dd(R, 1);
  if (lane == 0) t0 = {1.0, 0.0};
  const ddv t1 = dd_mul(t0, rho[0]);
  const ddv t2 = dd_mul(t1, rho[1]);
  ddv S = dd_add(dd_add(t0, t1), t2);
  const double j0 = 3.0 * lane;
  ddv W = dd_add(dd_add(dd_mul_d(t0, j0), dd_mul_d(t1, j0 + 1.0)), dd_mul_d(t2, j0 + 2.0));
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    S = dd_add(S, shfl_xor_dd(S, m));
    W = dd_add(W, shfl_xor_dd(W, m));
  }
  PD r;
  r.p = __shfl_sync(0xffffffffu, S.hi + S.lo, 0);
  r.dp = __shfl_sync(0xffffffffu, (ch / sh) * (W.hi + W.lo), 0);  // dP/dt = cot(t/2) sum_j j t_j
  return r;
}

// one warp per node k < kend (N sin theta*_k < 25, N > 64); every lane of the
// warp calls it with the same k
__device__ __forceinline__ void end_node(int64_t N, int64_t k, int lane, const NodeConst& K,
                                         double* __restrict__ theta, double* __restrict__ x,
                                         double* __restrict__ w, double* __restrict__ tN, int* __restrict__ status,
                                         int max_iter) {
  const double inv_Nh = K.inv_Nh;
  const double th0 = ((double)k + 0.75) * kPi * inv_Nh;
  double d = kJ0Zeros[k] * inv_Nh - th0;
  bool ok = false;
  double s = 0.0, c = 1.0, dp_final = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    double sh, ch;
    sincos(0.5 * (th0 + d), &sh, &ch);
    s = 2.0 * sh * ch;
    c = (ch - sh) * (ch + sh);
    const PD r = eval_series_warp(N, sh, ch, lane);
    const double step = r.p / r.dp;  // identical on every lane
    d -= step;
    if (!(fabs(d) < 1.0)) break;
    const double a_step = fabs(step);
    if (a_step * (double)N <= 1e-8 && (0.5 * fabs(c / s) + 1.0) * a_step * a_step * (double)N <= 1e-18) {
      dp_final = r.dp + step * ((c / s) * r.dp + (double)N * ((double)N + 1.0) * r.p);
      const double cn = c + s * step;
      s = s - c * step;
      c = cn;
      ok = true;
      break;
    }
  }
  if (lane != 0) return;
  if (!ok) atomicOr(status, 1);
  const double th = th0 + d;
  const double wk = 2.0 / (dp_final * dp_final);
  const double tk = kPi * (double)(N - 2 * k - 1) * (0.25 * inv_Nh) + (double)N * d;
  theta[k] = th;
  x[k] = c;
  w[k] = wk;
  tN[k] = tk;
  const int64_t km = N - 1 - k;
  theta[km] = kPi - th;
  x[km] = -c;
  w[km] = wk;
  tN[km] = -tk;
}

// One launch for every node: blocks [0, nbe) take the end nodes k < kend, one
// warp each (the dependent double-double series sets their length, so they
// start first and run under the interior nodes), blocks from nbe on the nodes
// kend <= k < ceil(N/2), one thread each.
constexpr int kNodeThreads = 128;
// work block b: the end nodes (b < nbe) or 128 interior nodes
__device__ __forceinline__ void node_block(int b, int64_t N, int64_t kend, int nbe, double CN, const HTab& H,
                                           const NodeConst& K, double* __restrict__ theta, double* __restrict__ x,
                                           double* __restrict__ w, double* __restrict__ tN,
                                           int* __restrict__ status, int max_iter) {
  if (b < nbe) {
    const int64_t k = (int64_t)b * (kNodeThreads / 32) + (threadIdx.x >> 5);
    if (k < kend) end_node(N, k, threadIdx.x & 31, K, theta, x, w, tN, status, max_iter);
    return;
  }
  const int64_t k = (int64_t)(b - nbe) * kNodeThreads + threadIdx.x;
  if (k >= (N + 1) / 2 || k < kend) return;
  interior_node(N, k, CN, H, K, theta, x, w, tN, status, max_iter);
}

// STRIDE: the grid is smaller than the nblocks blocks of work and every block
// strides over them (a node kernel run beside other kernels leaves part of each
// SM free); otherwise one block per work block.
template <bool STRIDE>
__global__ void __launch_bounds__(kNodeThreads) k_legpts(int64_t N, int64_t kend, int nbe, int nblocks, double CN,
                                                         HTab H, NodeConst K, double* __restrict__ theta,
                                                         double* __restrict__ x, double* __restrict__ w,
                                                         double* __restrict__ tN, int* __restrict__ status,
                                                         int max_iter) {
  if (!STRIDE) {
    node_block((int)blockIdx.x, N, kend, nbe, CN, H, K, theta, x, w, tN, status, max_iter);
    return;
  }
  for (int b = (int)blockIdx.x; b < nblocks; b += (int)gridDim.x)
    node_block(b, N, kend, nbe, CN, H, K, theta, x, w, tN, status, max_iter);
}

// nodes handled by end_node: the first k with N sin theta*_k >= 25 (at most 8)
int64_t end_nodes(int64_t N) {
  if (N <= 64) return 0;
  int64_t k = 0;
  while (k < kMaxEnds && (double)N * std::sin(((double)k + 0.75) * kPi / ((double)N + 0.5)) < 25.0) ++k;
  return k;
}

__global__ void k_dtheta(const double* __restrict__ tN, double* __restrict__ out, int64_t N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // exact for N a power of two (the FFT-based chain), correctly rounded otherwise
  if (k < N) out[k] = tN[k] / (double)N;
}

// h_{0,N} = 1, h_{m+1,N} = h_{m,N} (m+1/2)^2 / ((m+1)(N+m+3/2))
HTab htab(int64_t N) {
  HTab H;
  H.h[0] = 1.0;
  for (int m = 0; m + 1 < kMaxTerms; ++m)
    H.h[m + 1] = H.h[m] * (m + 0.5) * (m + 0.5) / ((m + 1.0) * ((double)N + m + 1.5));
  return H;
}

// the node kernel on `stream` (callers count the launch); max_grid > 0 caps the
// grid (the blocks stride over the work)
void launch_nodes(int64_t N, double CN, double* theta, double* x, double* w, double* tN, int* status,
                  cudaStream_t stream, int max_iter = kNodeIterMax, int max_grid = 0) {
  const int64_t kend = end_nodes(N);
  const int nbe = (int)((kend + kNodeThreads / 32 - 1) / (kNodeThreads / 32));
  const int64_t half = (N + 1) / 2;
  NodeConst K;
  const double Nh = (double)N + 0.5;
  K.inv_Nh = 1.0 / Nh;
  K.c1 = 0.125 / (Nh * ((double)N + 1.5));
  const int nblocks = (int)(nbe + (half + kNodeThreads - 1) / kNodeThreads);
  if (max_grid > 0 && max_grid < nblocks)
    k_legpts<true><<<(unsigned)max_grid, kNodeThreads, 0, stream>>>(N, kend, nbe, nblocks, CN, htab(N), K, theta,
                                                                    x, w, tN, status, max_iter);
  else
    k_legpts<false><<<(unsigned)nblocks, kNodeThreads, 0, stream>>>(N, kend, nbe, nblocks, CN, htab(N), K, theta,
                                                                     x, w, tN, status, max_iter);
}

}  // namespace

int launch_dtheta(Plan& P, double* out) {
  const int64_t N = P.p.N;
  k_dtheta<<<(unsigned)((N + 255) / 256), 256, 0, P.stream>>>(P.tN, out, N);
  launched(P, "dtheta", (double)N, 16.0 * N);
  return check_launch();
}

int launch_legpts(Plan& P, double CN, int blocks_per_sm) {
  const int64_t N = P.p.N;
  int grid = 0;
  if (blocks_per_sm > 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 1;
    }
    grid = blocks_per_sm * std::max(sms, 1);
  }
  launch_nodes(N, CN, P.theta, P.x, P.w, P.tN, P.status, P.stream, P.node_iter_max, grid);
  launched(P, "legpts", 0.0, 32.0 * N);
  return check_launch();
}

}  // namespace gbdlt

// ---------------------------------------------------------------------------
// Allocation-free node computation (gbdlt_legpts_noalloc)
//
// Some callers cannot allocate device memory where they need a quadrature
// rule: code that runs under a fixed, pre-reserved memory budget (an
// application whose own allocator owns every byte of the GPU), latency-critical
// paths where cudaMalloc's implicit device synchronisation is not acceptable,
// and plugins that are handed buffers by a host framework and may not call the
// CUDA allocator themselves.  For them this entry point computes the
// Gauss-Legendre rule without a plan: the node kernel's scratch (the scaled
// offsets t_k = N dtheta_k and the convergence status word) lives in a
// file-scope device array instead of a plan workspace, and the caller passes
// only the output buffers.
// ---------------------------------------------------------------------------
namespace gbdlt {
namespace {

constexpr int64_t kNoAllocMaxN = 65536;
// [0, kNoAllocMaxN): t_k; [kNoAllocMaxN, +32): status word (first int) and padding.
// 512 KB per GPU that loads the library, held until the process exits.
static __device__ __align__(256) double g_legpts_scratch[kNoAllocMaxN + 32];

// Device address of the scratch array in the current device's context.  Looked
// up on every call with that device current: a host-side reference to the
// symbol is not a device address, and an address kept from an earlier call
// would dangle once the context is destroyed (cudaDeviceReset, or the primary
// context released and made again), because the array then lives in the newly
// loaded module.  Once the module is loaded the lookup is a host-side query.
int scratch_on_current_device(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_legpts_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return GBDLT_ERR_CUDA;
  }
  *out = (double*)p;
  return GBDLT_OK;
}

// C_N = sqrt(4/pi) Gamma(N+1)/Gamma(N+3/2) by the running product
// C_{n+1} = C_n (n+1)/(n+3/2) in double-double, without allocating.
double cn_running(int64_t N) {
  double hi = 1.2732395447351628, lo = -7.871470670072994e-17;  // 4/pi
  for (int64_t n = 0; n < N; ++n) {
    const double b = (double)(n + 1);
    double p = hi * b;
    double e = std::fma(hi, b, -p);
    e = std::fma(lo, b, e);
    double s = p + e;
    lo = e - (s - p);
    hi = s;
    const double d = (double)n + 1.5;
    const double q1 = hi / d;
    const double pp = q1 * d;
    const double pe = std::fma(q1, d, -pp);
    const double r = ((hi - pp) - pe) + lo;
    const double q2 = r / d;
    hi = q1 + q2;
    lo = q2 - (hi - q1);
  }
  return hi + lo;
}

}  // namespace

}  // namespace gbdlt

extern "C" int gbdlt_legpts_noalloc(int64_t N, double* x, double* theta, double* w, double* dtheta,
                                    void* cuda_stream) {
  using namespace gbdlt;
  if (N < 1 || N > kNoAllocMaxN) return GBDLT_ERR_UNSUPPORTED_N;
  if (!x || !theta || !w) return GBDLT_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  double* scratch = nullptr;
  int st = scratch_on_current_device(&scratch);
  if (st) return st;
  double* tN = scratch;
  int* status = reinterpret_cast<int*>(scratch + kNoAllocMaxN);
  // the status word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(status, 0, sizeof(int), stream) != cudaSuccess) {
    cudaGetLastError();
    return GBDLT_ERR_CUDA;
  }
  launch_nodes(N, cn_running(N), theta, x, w, tN, status, stream);
  count_launch();
  if (dtheta) {
    k_dtheta<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(tN, dtheta, N);
    count_launch();
  }
  if (check_launch()) return GBDLT_ERR_CUDA;
  int hs = 0;
  if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return GBDLT_ERR_CUDA;
  }
  return (hs & 1) ? GBDLT_ERR_NOT_CONVERGED : GBDLT_OK;
}
