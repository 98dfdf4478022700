// Batched complex FFT of power-of-two length N on one GPU.
//
// This is the transform engine behind every DCT/DST of the method (Sec. 2.3,
// Eq. 13; the DCT/DST are reduced to complex FFTs of length N by the pre- and
// post-processing kernels in stages.cu).  Sign convention: DIR = +1 computes
// y_k = sum_n x_n e^{+2 pi i nk/N}, DIR = -1 the conjugate kernel; no scaling.
//
// Layout: nvec vectors, each N contiguous complex values (float2/double2).
//  * N <= 4096: one pass; a CTA holds 4096/N vectors in shared memory and runs
//    an in-place Stockham autosort FFT: one radix-2/4/8 stage for log2 N mod 4,
//    then radix-16 stages whose 16-point DFTs run in registers (4 x 4 with
//    constant internal twiddles), so L = 1024 takes 3 shared-memory passes.
//    Shared memory holds element i of a line at i + i/16 (one pad element per
//    16, one per line) so the stride-16 stores of a radix-16 stage spread over
//    all banks.
//  * N > 4096: four-step with N = L1 * L2 (L1, L2 <= 4096).  Pass 1 ("columns"):
//    a CTA loads C = 4096/L1 adjacent columns n2 (C contiguous elements per
//    row, so global loads and stores are coalesced segments), transforms along
//    n1, multiplies by e^{DIR 2 pi i n2 k1 / N} and stores in place.  Pass 2
//    ("rows"): a CTA loads C2 = 4096/L2 contiguous rows k1, transforms along
//    n2 and stores X[k1 + L1 k2] into the second buffer, C2 contiguous elements
//    per k2.
// Twiddles come from tables (no trigonometry in the hot loop): the inner
// Stockham twiddles from a 4096-entry table e^{2 pi i j/4096}, the inter-pass
// twiddle from a table of e^{2 pi i e/N} (one entry per e in FP64; in FP32 the
// product of a two-level table).
//
// FP64 stages with twiddles (radix 16, Ns > 1) are written for GB300's FP64
// pipe, which retires two operations per SM per clock while every other pipe
// is idle: each radix-16 butterfly is two layers of radix-4 decimation-in-time
// butterflies whose twiddle products are folded into fused multiply-adds in the
// cosine/tangent form of Linzer and Feig (IBM J. Res. Dev., 1993):
//   w b = sigma * ((b_x - tau b_y) + i (b_y + tau b_x)),  sigma = cos, tau = tan,
// or, where |sin| > |cos|, the same with sigma = sin, tau = cot on the swapped
// components of b (the swap is a register select, not an FP64 operation).  A
// radix-4 butterfly with twiddle U,
//   y_q = sum_r omega_4^{rq} U^r a_r
//       = (a0 +- U^2 a2) + omega_4^q U (a1 +- U^2 a3),
// then costs 24 FMAs for 4 points, against 16 additions and 3 complex products
// (28 operations) in the plain form; a twiddled radix-16 stage drops from
// 13.75 to 12 FP64 operations per point.
#include <algorithm>
#include <mutex>
#include <vector>

#include <cuda.h>  // CUtensorMap (types only; the encoder is fetched from the driver at run time)

#include "gbdlt_internal.cuh"

namespace gbdlt {

constexpr int FFT_TILE = 4096;
constexpr int FFT_THREADS = 256;
// largest tile footprint in elements: lines * (L + L/16 + 1) with lines * L = 4096
constexpr int FFT_SMEM_ELEMS = FFT_TILE + FFT_TILE / 16 + 256;

// Shared-memory index of element i of line `line`: one pad element every 16
// (stride-16 butterfly stores then hit distinct banks) and one per line.
__device__ __forceinline__ int sidx(int line, int LP, int i) { return line * LP + i + (i >> 4); }
__host__ __device__ __forceinline__ int line_pitch(int L) { return L + (L >> 4) + (L >= 16 ? 1 : 0); }

// e^{2 pi i e / N} from the two-level table, multiplied in the precision T
template <typename T>
__device__ __forceinline__ C2<T> tw_lookup(const C2<T>* __restrict__ hi, const C2<T>* __restrict__ lo,
                                           int64_t e) {
  return cmul<T>(hi[e >> 12], lo[e & 4095]);
}

// e^{2 pi i e / N} in FP32 for 0 <= e < N <= 2^24, N a power of two: sincospif
// of the argument 2e/N, which is exact in float (e fits the significand and 2/N
// is a power of two), so the only rounding is the function's own (no table
// loads: the FP32 passes are bound by the latency of their global loads)
__device__ __forceinline__ C2<float> tw_pow2_f32(int64_t e, float two_over_n) {
  float s, c;
  sincospif((float)e * two_over_n, &s, &c);
  return mk<float>(c, s);
}

// multiply by e^{DIR i a} given (cos a, sin a)
template <typename T, int DIR>
__device__ __forceinline__ C2<T> rot(C2<T> v, T c, T s) {
  const T sd = DIR > 0 ? s : -s;
  return cmul<T>(v, mk<T>(c, sd));
}

template <typename T>
__device__ __forceinline__ T shfl_xor_t(T v, int m) {
  if constexpr (std::is_same<T, ffd>::value) {
    return ffd(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
  } else {
    return __shfl_xor_sync(0xffffffffu, v, m);
  }
}

// kernel names for the profiler: FP64, FP32 and float-float launches apart
template <typename T>
constexpr const char* kname(const char* d, const char* f, const char* ff) {
  return is_f64<T> ? d : is_f32<T> ? f : ff;
}

// ---------------------------------------------------------------- cosine/tangent twiddles (FP64)
// Table entry for angle a: (sx, sy, t, swap) with, if |cos a| >= |sin a|,
// sx = sy = cos a, t = tan a, swap = 0; otherwise sx = -sin a, sy = sin a,
// t = cot a, swap = 1.  Then e^{ia} b = (sx R_x, sy R_y) with
// R = (b'_x - t b'_y, b'_y + t b'_x), b' = b or (b_y, b_x) if swap.
struct LFTw {
  double sx, sy, t;
  bool sw;
};

__device__ __forceinline__ LFTw lf_load(const double2* __restrict__ tab, int e) {
  const double2 a = tab[2 * e], b = tab[2 * e + 1];
  return {a.x, a.y, b.x, __double_as_longlong(b.y) != 0};
}

__device__ __forceinline__ C2<double> lf_rot(const LFTw& T, const C2<double> b) {
  const double bx = T.sw ? b.y : b.x;
  const double by = T.sw ? b.x : b.y;
  return mk<double>(fma(-T.t, by, bx), fma(T.t, bx, by));
}

// in place: a_q <- sum_r omega_4^{rq} U^r a_r, omega_4 = e^{DIR i pi/2}; U2 = U^2
template <int DIR>
__device__ __forceinline__ void lf_dft4(C2<double>& a0, C2<double>& a1, C2<double>& a2, C2<double>& a3,
                                        const LFTw& U, const LFTw& U2) {
  using CD = C2<double>;
  const CD r2 = lf_rot(U2, a2), r3 = lf_rot(U2, a3);
  const CD b0 = mk<double>(fma(U2.sx, r2.x, a0.x), fma(U2.sy, r2.y, a0.y));   // a0 + U^2 a2
  const CD b1 = mk<double>(fma(-U2.sx, r2.x, a0.x), fma(-U2.sy, r2.y, a0.y)); // a0 - U^2 a2
  const CD c0 = mk<double>(fma(U2.sx, r3.x, a1.x), fma(U2.sy, r3.y, a1.y));   // a1 + U^2 a3
  const CD c1 = mk<double>(fma(-U2.sx, r3.x, a1.x), fma(-U2.sy, r3.y, a1.y)); // a1 - U^2 a3
  const CD q0 = lf_rot(U, c0), q1 = lf_rot(U, c1);
  a0 = mk<double>(fma(U.sx, q0.x, b0.x), fma(U.sy, q0.y, b0.y));    // b0 + U c0
  a2 = mk<double>(fma(-U.sx, q0.x, b0.x), fma(-U.sy, q0.y, b0.y));  // b0 - U c0
  // b1 +- omega_4 U c1 with omega_4 (p + iq) = DIR (-q + ip)
  if (DIR > 0) {
    a1 = mk<double>(fma(-U.sy, q1.y, b1.x), fma(U.sx, q1.x, b1.y));
    a3 = mk<double>(fma(U.sy, q1.y, b1.x), fma(-U.sx, q1.x, b1.y));
  } else {
    a1 = mk<double>(fma(U.sy, q1.y, b1.x), fma(-U.sx, q1.x, b1.y));
    a3 = mk<double>(fma(-U.sy, q1.y, b1.x), fma(U.sx, q1.x, b1.y));
  }
}

// Radix-16 DIT butterfly with twiddles w^{r k}, w = e^{DIR 2 pi i/(16 Ns)}, as two
// radix-4 layers (r = r1 + 4 r2, q = q1 + 4 q2):
//   B_r1(q1)   = sum_r2 omega_4^{r2 q1} W^{r2} x_{r1+4r2},          W = w^{4k}
//   y_{q1+4q2} = sum_r1 omega_4^{r1 q2} V_q1^{r1} B_r1(q1),  V_q1 = w^{k + Ns q1}
// On return v[4 q1 + q2] holds y_{q1 + 4 q2}.
template <int DIR>
__device__ __forceinline__ void lf_dft16(C2<double>* v, const double2* __restrict__ lf, int k, int Ns) {
  const int s4 = 1024 / Ns;  // 4096 / (4 Ns): table step of w^4
  const int s16 = 256 / Ns;  // 4096 / (16 Ns): table step of w
  const LFTw W = lf_load(lf, k * s4), W2 = lf_load(lf, 2 * k * s4);
#pragma unroll
  for (int r1 = 0; r1 < 4; ++r1) lf_dft4<DIR>(v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12], W, W2);
#pragma unroll
  for (int q1 = 0; q1 < 4; ++q1) {
    int e = (k + Ns * q1) * s16;
    // tie the table index to the data just computed so that the compiler loads
    // each twiddle pair when it is needed instead of holding all of them in
    // registers (the 16 values already take 64)
    asm volatile("" : "+r"(e) : "d"(v[4 * q1].x));
    const LFTw V = lf_load(lf, e), V2 = lf_load(lf, 2 * e);
    lf_dft4<DIR>(v[4 * q1], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3], V, V2);
  }
}

// ---------------------------------------------------------------- small DFTs in registers
template <typename T, int DIR>
__device__ __forceinline__ void dft4(C2<T>& a0, C2<T>& a1, C2<T>& a2, C2<T>& a3) {
  const C2<T> s02 = cadd<T>(a0, a2), d02 = csub<T>(a0, a2);
  const C2<T> s13 = cadd<T>(a1, a3), d13 = cmul_i<T, DIR>(csub<T>(a1, a3));
  a0 = cadd<T>(s02, s13);
  a1 = cadd<T>(d02, d13);
  a2 = csub<T>(s02, s13);
  a3 = csub<T>(d02, d13);
}

template <typename T, int DIR>
__device__ __forceinline__ void dft2(C2<T>* v) {
  const C2<T> a = v[0], b = v[1];
  v[0] = cadd<T>(a, b);
  v[1] = csub<T>(a, b);
}

template <typename T, int DIR>
__device__ __forceinline__ void dft4v(C2<T>* v) {
  dft4<T, DIR>(v[0], v[1], v[2], v[3]);
}

// 8 = 2 x 4: E = DFT4(even), O = DFT4(odd), y_k = E_k + w8^k O_k, y_{k+4} = E_k - w8^k O_k
template <typename T, int DIR>
__device__ __forceinline__ void dft8(C2<T>* v) {
  const T h = (T)0.70710678118654752440;
  C2<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C2<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<T, DIR>(e0, e1, e2, e3);
  dft4<T, DIR>(o0, o1, o2, o3);
  o1 = rot<T, DIR>(o1, h, h);
  o2 = cmul_i<T, DIR>(o2);
  o3 = rot<T, DIR>(o3, -h, h);
  v[0] = cadd<T>(e0, o0);
  v[4] = csub<T>(e0, o0);
  v[1] = cadd<T>(e1, o1);
  v[5] = csub<T>(e1, o1);
  v[2] = cadd<T>(e2, o2);
  v[6] = csub<T>(e2, o2);
  v[3] = cadd<T>(e3, o3);
  v[7] = csub<T>(e3, o3);
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2:
// B[n2][k1] = DFT4_n1(x[4 n1 + n2]),  B *= w16^{n2 k1},  y[k1 + 4 k2] = DFT4_n2(B[n2][k1])
template <typename T, int DIR>
__device__ __forceinline__ void dft16(C2<T>* v) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // 2 pi / 16
  const T h = (T)0.70710678118654752440;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<T, DIR>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // now v[n2 + 4 k1] = B[n2][k1]; twiddles w16^{n2 k1}
  v[1 + 4 * 1] = rot<T, DIR>(v[1 + 4 * 1], c1, s1);   // e = 1
  v[1 + 4 * 2] = rot<T, DIR>(v[1 + 4 * 2], h, h);     // e = 2
  v[1 + 4 * 3] = rot<T, DIR>(v[1 + 4 * 3], s1, c1);   // e = 3
  v[2 + 4 * 1] = rot<T, DIR>(v[2 + 4 * 1], h, h);     // e = 2
  v[2 + 4 * 2] = cmul_i<T, DIR>(v[2 + 4 * 2]);        // e = 4
  v[2 + 4 * 3] = rot<T, DIR>(v[2 + 4 * 3], -h, h);    // e = 6
  v[3 + 4 * 1] = rot<T, DIR>(v[3 + 4 * 1], s1, c1);   // e = 3
  v[3 + 4 * 2] = rot<T, DIR>(v[3 + 4 * 2], -h, h);    // e = 6
  v[3 + 4 * 3] = rot<T, DIR>(v[3 + 4 * 3], -c1, -s1); // e = 9
  C2<T> y[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C2<T> a0 = v[0 + 4 * k1], a1 = v[1 + 4 * k1], a2 = v[2 + 4 * k1], a3 = v[3 + 4 * k1];
    dft4<T, DIR>(a0, a1, a2, a3);
    y[k1] = a0;
    y[k1 + 4] = a1;
    y[k1 + 8] = a2;
    y[k1 + 12] = a3;
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = y[r];
}

template <typename T, int DIR, int R>
__device__ __forceinline__ void dftR(C2<T>* v) {
  if constexpr (R == 2) dft2<T, DIR>(v);
  if constexpr (R == 4) dft4v<T, DIR>(v);
  if constexpr (R == 8) dft8<T, DIR>(v);
  if constexpr (R == 16) dft16<T, DIR>(v);
}

// FP64 radix-16 Stockham stage with Ns > 1 on the fused cosine/tangent form
template <int DIR>
__device__ __forceinline__ void stage_lf16(C2<double>* sm, int L, int logL, int lines, int LP, int Ns,
                                           const double2* __restrict__ lf) {
  using CD = C2<double>;
  constexpr int PER = FFT_TILE / 16 / FFT_THREADS;
  const int LR = L >> 4;
  const int logLR = logL - 4;
  const int nbf = lines * LR;
  CD v[PER][16];
  int dst[PER], ln[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * FFT_THREADS;
    dst[q] = -1;
    if (b < nbf) {
      const int line = b >> logLR;
      const int j = b & (LR - 1);
      const int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < 16; ++r) v[q][r] = sm[sidx(line, LP, j + r * LR)];
      lf_dft16<DIR>(v[q], lf, k, Ns);
      ln[q] = line;
      dst[q] = (j - k) * 16 + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (dst[q] >= 0) {
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) sm[sidx(ln[q], LP, dst[q] + (q1 + 4 * q2) * Ns)] = v[q][4 * q1 + q2];
    }
  }
  __syncthreads();
}

// One Stockham stage of radix R over `lines` vectors of length L (current
// sub-transform length Ns): butterfly j reads x[j + r L/R], applies
// w_{Ns R}^{r (j mod Ns)}, takes the R-point DFT and writes
// y[(j / Ns) Ns R + (j mod Ns) + r Ns].  Twiddles come from the 4096-entry
// table; in FP32 only the power-of-two multiples are loaded and the rest are
// products of them (FP32 arithmetic is cheap, table traffic is not).
template <typename T, int DIR, int R>
__device__ __forceinline__ void stage(C2<T>* sm, int L, int logL, int lines, int LP, int Ns,
                                      const C2<T>* __restrict__ tw, const double2* __restrict__ lf) {
  using CT = C2<T>;
  constexpr int PER = FFT_TILE / R / FFT_THREADS;
  const int LR = L / R;
  const int logLR = logL - (R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4);
  const int nbf = lines * LR;
  CT v[PER][R];
  int dst[PER], ln[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * FFT_THREADS;
    dst[q] = -1;
    if (b < nbf) {
      const int line = b >> logLR;
      const int j = b & (LR - 1);
      const int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = sm[sidx(line, LP, j + r * LR)];
      if (Ns > 1) {
        const int step = FFT_TILE / (Ns * R);
        CT w[R];
#pragma unroll
        for (int r = 1; r < R; ++r) {
          if (!is_f32<T> || (r & (r - 1)) == 0) {
            w[r] = tw[r * k * step];
          } else {
            w[r] = cmul<T>(w[r & (r - 1)], w[r & -r]);
          }
        }
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul<T>(v[q][r], mk<T>(w[r].x, DIR > 0 ? w[r].y : -w[r].y));
      }
      ln[q] = line;
      dst[q] = (j - k) * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    if (dst[q] >= 0) {
      dftR<T, DIR, R>(v[q]);
#pragma unroll
      for (int r = 0; r < R; ++r) sm[sidx(ln[q], LP, dst[q] + r * Ns)] = v[q][r];
    }
  }
  __syncthreads();
}

// Global -> shared tile load, thread i taking elements i, i + 256, ...  Every
// thread issues a batch of loads into registers before it stores them, so each
// thread keeps several global loads in flight: all 16 of its elements in FP32
// (those passes are bound by global-load latency), 8 in FP64 and float-float,
// whose butterflies need the registers only after the load phase.
template <typename T, typename Idx, typename Ld>
__device__ __forceinline__ void load_tile(C2<T>* sm, int tot, Idx sidx_of, Ld ld) {
  constexpr int B = is_f32<T> ? FFT_TILE / FFT_THREADS : 8;
  for (int i0 = 0; i0 < tot; i0 += B * FFT_THREADS) {
    C2<T> r[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int i = i0 + threadIdx.x + q * FFT_THREADS;
      if (i < tot) r[q] = ld(i);
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int i = i0 + threadIdx.x + q * FFT_THREADS;
      if (i < tot) sm[sidx_of(i)] = r[q];
    }
  }
}

// In-place FFT of `lines` vectors of length L held at sidx(line, LP, i):
// one stage of radix 2^(log2 L mod 4) (if any), then radix-16 stages.
template <typename T, int DIR>
__device__ void fft_tile(C2<T>* sm, int L, int logL, int lines, int LP, const C2<T>* __restrict__ tw,
                         const double2* __restrict__ lf) {
  int Ns = 1;
  const int rem = logL & 3;
  if (rem == 1) {
    stage<T, DIR, 2>(sm, L, logL, lines, LP, Ns, tw, lf);
    Ns = 2;
  } else if (rem == 2) {
    stage<T, DIR, 4>(sm, L, logL, lines, LP, Ns, tw, lf);
    Ns = 4;
  } else if (rem == 3) {
    stage<T, DIR, 8>(sm, L, logL, lines, LP, Ns, tw, lf);
    Ns = 8;
  }
  if constexpr (is_f64<T>) {
    // FP64: the untwiddled first radix-16 stage, then the fused cosine/tangent stages
    if (Ns == 1 && Ns < L) {
      stage<T, DIR, 16>(sm, L, logL, lines, LP, 1, tw, lf);
      Ns = 16;
    }
    while (Ns < L) {
      stage_lf16<DIR>(reinterpret_cast<C2<double>*>(sm), L, logL, lines, LP, Ns, lf);
      Ns <<= 4;
    }
  } else {
    while (Ns < L) {
      stage<T, DIR, 16>(sm, L, logL, lines, LP, Ns, tw, lf);
      Ns <<= 4;
    }
  }
}

// Launch-local vector j -> vector (j / count) * stride + first + j % count of the
// buffer: a launch can cover, for every batch item, a contiguous run of the
// item's vectors (the bands the pruned kernels do not take).
struct VecMap {
  int64_t first, count, stride;
};
__device__ __forceinline__ int64_t vec_of(const VecMap& m, int64_t j) {
  return (j / m.count) * m.stride + m.first + j % m.count;
}
inline int64_t vec_of_host(const VecMap& m, int64_t j) { return (j / m.count) * m.stride + m.first + j % m.count; }

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS, is_f32<T> ? 4 : 2)
    k_fft_single(C2<T>* __restrict__ data, int L, int logL, int64_t nvec, const C2<T>* __restrict__ tw4096,
                 const double2* __restrict__ lf) {
  extern __shared__ unsigned char smraw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int lines_max = FFT_TILE / L;
  const int64_t v0 = (int64_t)blockIdx.x * lines_max;
  const int lines = (int)min((int64_t)lines_max, nvec - v0);
  const int LP = line_pitch(L);
  const int tot = lines * L;
  C2<T>* g = data + v0 * L;
  load_tile<T>(sm, tot, [&](int i) { return sidx(i >> logL, LP, i & (L - 1)); }, [&](int i) { return g[i]; });
  __syncthreads();
  fft_tile<T, DIR>(sm, L, logL, lines, LP, tw4096, lf);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) g[i] = sm[sidx(i >> logL, LP, i & (L - 1))];
}

// column pass of tile bx (C columns) of launch-local vector by
template <typename T, int DIR>
__device__ __forceinline__ void fft_cols_tile(unsigned char* smraw, C2<T>* __restrict__ data, int64_t N, int L1,
                                              int logL1, int L2, int C, int logC,
                                              const C2<T>* __restrict__ tw4096, const C2<T>* __restrict__ thi,
                                              const C2<T>* __restrict__ tlo, const C2<T>* __restrict__ tfull,
                                              const double2* __restrict__ lf, VecMap vm, int bx, int64_t by) {
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int c0 = bx * C;
  C2<T>* g = data + vec_of(vm, by) * N;
  const int LP = line_pitch(L1);
  const int tot = L1 * C;
  load_tile<T>(sm, tot, [&](int i) { return sidx(i & (C - 1), LP, i >> logC); },
               [&](int i) { return g[(int64_t)(i >> logC) * L2 + c0 + (i & (C - 1))]; });
  __syncthreads();
  fft_tile<T, DIR>(sm, L1, logL1, C, LP, tw4096, lf);
#pragma unroll 4
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    const int k1 = i >> logC, c = i & (C - 1);
    const int64_t e = (int64_t)(c0 + c) * k1;
    C2<T> val = sm[sidx(c, LP, k1)];
    if (e != 0) {
      // FP64 and float-float: one table entry per e; FP32: product of the two-level entries
      const C2<T> w = !is_f32<T> ? tfull[e] : tw_lookup<T>(thi, tlo, e);
      val = cmul<T>(val, mk<T>(w.x, DIR > 0 ? w.y : -w.y));
    }
    g[(int64_t)k1 * L2 + c0 + c] = val;
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS, is_f32<T> ? 4 : 2)
    k_fft_cols(C2<T>* __restrict__ data, int64_t N, int L1, int logL1, int L2, int C, int logC,
               const C2<T>* __restrict__ tw4096, const C2<T>* __restrict__ thi,
               const C2<T>* __restrict__ tlo, const C2<T>* __restrict__ tfull, const double2* __restrict__ lf,
               VecMap vm) {
  extern __shared__ unsigned char smraw[];
  fft_cols_tile<T, DIR>(smraw, data, N, L1, logL1, L2, C, logC, tw4096, thi, tlo, tfull, lf, vm, (int)blockIdx.x,
                        (int64_t)blockIdx.y);
}

// row pass of tile bx (C2n rows) of launch-local vector by
template <typename T, int DIR>
__device__ __forceinline__ void fft_rows_tile(unsigned char* smraw, const C2<T>* __restrict__ in,
                                              C2<T>* __restrict__ out, int64_t N, int L1, int L2, int logL2,
                                              int C2n, int logC2, const C2<T>* __restrict__ tw4096,
                                              const double2* __restrict__ lf, VecMap vm, int bx, int64_t by) {
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int r0 = bx * C2n;
  const int64_t v = vec_of(vm, by);
  const C2<T>* g = in + v * N;
  C2<T>* o = out + v * N;
  const int LP = line_pitch(L2);
  const int tot = L2 * C2n;
  load_tile<T>(sm, tot, [&](int i) { return sidx(i >> logL2, LP, i & (L2 - 1)); },
               [&](int i) { return g[(int64_t)(r0 + (i >> logL2)) * L2 + (i & (L2 - 1))]; });
  __syncthreads();
  fft_tile<T, DIR>(sm, L2, logL2, C2n, LP, tw4096, lf);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    const int k2 = i >> logC2, line = i & (C2n - 1);
    o[(int64_t)(r0 + line) + (int64_t)L1 * k2] = sm[sidx(line, LP, k2)];
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS, is_f32<T> ? 4 : 2)
    k_fft_rows(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, int64_t N, int L1, int L2,
               int logL2, int C2n, int logC2, const C2<T>* __restrict__ tw4096,
               const double2* __restrict__ lf, VecMap vm) {
  extern __shared__ unsigned char smraw[];
  fft_rows_tile<T, DIR>(smraw, in, out, N, L1, L2, logL2, C2n, logC2, tw4096, lf, vm, (int)blockIdx.x,
                        (int64_t)blockIdx.y);
}

// Mixed passes: the FP64 and the float-float vectors of one stage in one launch.
// On GB300 the FP64 and FP32 pipes are separate; a CTA of each kind on an SM
// (the two kinds use the same registers and shared memory per CTA) keeps both
// busy, where two launches on two streams run mostly one after the other (the
// first launch's CTAs fill every SM).  CTA b takes, while both kinds have
// tiles left, an FP64 tile for even b and a float-float tile for odd b; then the
// tiles of the kind with more.  Tile t of a kind is column (row) block
// t mod nx of launch-local vector t / nx.
struct MixArgs {
  C2<double>* a64;
  C2<double>* b64;
  ffc* aff;
  ffc* bff;
  int64_t n64, nff;  // tiles of each kind
  VecMap vm64, vmff;
};
__device__ __forceinline__ bool mix_pick(const MixArgs& M, int64_t b, int64_t& t) {
  const int64_t both = 2 * min(M.n64, M.nff);
  if (b < both) {
    t = b >> 1;
    return (b & 1) == 0;
  }
  t = b - both / 2;
  return M.n64 > M.nff;
}

template <int DIR>
__global__ void __launch_bounds__(FFT_THREADS, 2)
    k_fft_cols_mix(MixArgs M, int64_t N, int L1, int logL1, int L2, int C, int logC, int nx,
                   const double2* __restrict__ tw64, const double2* __restrict__ full64,
                   const double2* __restrict__ lf, const ffc* __restrict__ twff, const ffc* __restrict__ fullff) {
  extern __shared__ unsigned char smraw[];
  int64_t t;
  if (mix_pick(M, blockIdx.x, t))
    fft_cols_tile<double, DIR>(smraw, M.a64, N, L1, logL1, L2, C, logC, tw64, nullptr, nullptr, full64, lf, M.vm64,
                               (int)(t % nx), t / nx);
  else
    fft_cols_tile<ffd, DIR>(smraw, M.aff, N, L1, logL1, L2, C, logC, twff, nullptr, nullptr, fullff, nullptr,
                            M.vmff, (int)(t % nx), t / nx);
}

template <int DIR>
__global__ void __launch_bounds__(FFT_THREADS, 2)
    k_fft_rows_mix(MixArgs M, int64_t N, int L1, int L2, int logL2, int C2n, int logC2, int nx,
                   const double2* __restrict__ tw64, const double2* __restrict__ lf, const ffc* __restrict__ twff) {
  extern __shared__ unsigned char smraw[];
  int64_t t;
  if (mix_pick(M, blockIdx.x, t))
    fft_rows_tile<double, DIR>(smraw, M.a64, M.b64, N, L1, L2, logL2, C2n, logC2, tw64, lf, M.vm64,
                               (int)(t % nx), t / nx);
  else
    fft_rows_tile<ffd, DIR>(smraw, M.aff, M.bff, N, L1, L2, logL2, C2n, logC2, twff, nullptr, M.vmff,
                            (int)(t % nx), t / nx);
}

// ---------------------------------------------------------------- pruned passes
// A band of rows [ka, kb) (and their mirrors) reads the forward transform only at
// the bins of two windows, |y| < R and |y - N/2| < R cyclically (R = kb/2 + 2),
// and its transposed transform has nonzero input only there.  With the four-step
// split y = k1 + L1 k2 (forward) and n = n1 L2 + n2 (input), and 2R <= L1, L2:
//  * forward: row k1 < R needs k2 in {0, L2/2}, row k1 >= L1 - R needs
//    k2 in {L2 - 1, L2/2 - 1}, other rows nothing: each needed row is two even/odd
//    sums (twiddled by e^{-DIR 2 pi i n2/L2} for the high rows) instead of an FFT;
//  * transposed: column n2 < R has input only at n1 in {0, L1/2}, column
//    n2 >= L2 - R only at n1 in {L1/2 - 1, L1 - 1}, other columns none: the column
//    transform is x_a +- x_b times one twiddle, w_N^{n2 k1} or w_N^{k1 (n2 - L2)}.

// forward: one warp per needed row, 8 rows per CTA; grid (ceil(2R / 8), vectors)
template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_rows_pruned(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, int64_t N, int L1, int L2, int R,
                      const C2<T>* __restrict__ tw4096, VecMap vm) {
  const int r = blockIdx.x * (FFT_THREADS / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= 2 * R) return;  // whole warp
  const bool low = r < R;
  const int k1 = low ? r : L1 - 2 * R + r;
  const int64_t v = vec_of(vm, blockIdx.y);
  const C2<T>* g = in + v * N + (int64_t)k1 * L2;
  C2<T>* o = out + v * N;
  const int step = FFT_TILE / L2;
  T ex = 0, ey = 0, ox = 0, oy = 0;
  for (int n2 = 2 * lane; n2 < L2; n2 += 64) {
    C2<T> a = g[n2], b = g[n2 + 1];
    if (!low) {
      // times e^{-DIR 2 pi i n2 / L2}
      const C2<T> wa = tw4096[n2 * step], wb = tw4096[(n2 + 1) * step];
      a = cmul<T>(a, mk<T>(wa.x, DIR > 0 ? -wa.y : wa.y));
      b = cmul<T>(b, mk<T>(wb.x, DIR > 0 ? -wb.y : wb.y));
    }
    ex += a.x;
    ey += a.y;
    ox += b.x;
    oy += b.y;
  }
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    ex += shfl_xor_t(ex, m);
    ey += shfl_xor_t(ey, m);
    ox += shfl_xor_t(ox, m);
    oy += shfl_xor_t(oy, m);
  }
  if (lane == 0) {
    const int64_t ka = low ? 0 : L2 - 1, kb = low ? L2 / 2 : L2 / 2 - 1;
    o[k1 + (int64_t)L1 * ka] = mk<T>(ex + ox, ey + oy);
    o[k1 + (int64_t)L1 * kb] = mk<T>(ex - ox, ey - oy);
  }
}

// transposed: grid (L2 / C column groups, vectors), in place
template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_cols_pruned(C2<T>* __restrict__ data, int64_t N, int L1, int L2, int R, int C, int logC,
                      const C2<T>* __restrict__ thi, const C2<T>* __restrict__ tlo,
                      const C2<T>* __restrict__ tfull, VecMap vm) {
  __shared__ C2<T> xs[2][64];  // C <= 4096 / L1 <= 64 (L1 >= 64 when N > 4096)
  const int c0 = blockIdx.x * C;
  C2<T>* g = data + vec_of(vm, blockIdx.y) * N;
  for (int c = threadIdx.x; c < C; c += FFT_THREADS) {
    const int n2 = c0 + c;
    C2<T> a = mk<T>(0, 0), b = mk<T>(0, 0);
    if (n2 < R) {
      a = g[n2];
      b = g[(int64_t)(L1 / 2) * L2 + n2];
    } else if (n2 >= L2 - R) {
      a = g[(int64_t)(L1 - 1) * L2 + n2];
      b = g[(int64_t)(L1 / 2 - 1) * L2 + n2];
    }
    xs[0][c] = a;
    xs[1][c] = b;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L1 * C; i += FFT_THREADS) {
    const int k1 = i >> logC, c = i & (C - 1);
    const int n2 = c0 + c;
    C2<T> val = mk<T>(0, 0);
    const bool lowc = n2 < R;
    if (lowc || n2 >= L2 - R) {
      const C2<T> a = xs[0][c], b = xs[1][c];
      val = (k1 & 1) ? csub<T>(a, b) : cadd<T>(a, b);
      const int64_t e = lowc ? (int64_t)n2 * k1 : (N - (int64_t)k1 * (L2 - n2)) & (N - 1);
      if (e != 0) {
        const C2<T> w = !is_f32<T> ? tfull[e] : tw_lookup<T>(thi, tlo, e);
        val = cmul<T>(val, mk<T>(w.x, DIR > 0 ? w.y : -w.y));
      }
    }
    g[(int64_t)k1 * L2 + n2] = val;
  }
}

// ---------------------------------------------------------------- FP32 passes, compile-time lines
// The FP32 passes issue every instruction the FP32 pipe does not hide, and in the
// generic stage most of them are shared-memory index arithmetic (line length and
// sub-transform length are run-time values there).  These kernels take log2 of
// the line length as a template parameter: the stage sequence, strides and masks
// are constants, the 16 elements of a butterfly sit at immediate offsets from
// one base whenever the stride is a multiple of 16, and the tile is always full
// (four-step passes), so no bounds tests remain.
__host__ __device__ constexpr int line_pitch_ct(int L) { return L + (L >> 4) + (L >= 16 ? 1 : 0); }

// Twiddles: with R0 = 0, tw is the 4096-entry global table e^{2 pi i j/4096};
// with R0 > 0 (the radix of the line's first stage), tw is the shared-memory
// table of tw_fill: for each twiddled radix-16 stage (sub-transform length NS =
// R0, 16 R0, ...) four rows of NS entries, row b holding the twiddles of
// r = 2^b, w^{r k} for k < NS, so that the lanes of a warp read consecutive
// entries (the same rounded values as the global table)
template <int DIR, int R, int LOGL, int LOGNS, int R0 = 0>
__device__ __forceinline__ void stage_ct(C2<float>* sm, const C2<float>* __restrict__ tw) {
  using CT = C2<float>;
  constexpr int L = 1 << LOGL;
  constexpr int LOGR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
  constexpr int LR = L / R, LOGLR = LOGL - LOGR;
  constexpr int NS = 1 << LOGNS;
  constexpr int LP = line_pitch_ct(L);
  constexpr int PER = FFT_TILE / R / FFT_THREADS;
  constexpr int SRD = LR + (LR >> 4), SWR = NS + (NS >> 4);
  CT v[PER][R];
  int lnq[PER], dq[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * FFT_THREADS;
    const int line = b >> LOGLR;
    const int j = b & (LR - 1);
    const int k = j & (NS - 1);
    if constexpr ((LR & 15) == 0) {
      const CT* p = sm + line * LP + j + (j >> 4);
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = p[r * SRD];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = sm[sidx(line, LP, j + r * LR)];
    }
    if constexpr (NS > 1) {
      const int ks = k * (FFT_TILE / (NS * R));
      // rows of this stage's shared table (R0 > 0: 4 (NS - R0) / 15 entries precede)
      const C2<float>* ts = tw + (R0 > 0 ? 4 * (NS - R0) / 15 : 0);
      CT w[R];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        if ((r & (r - 1)) == 0) {
          if constexpr (R0 > 0) {
            w[r] = ts[(r == 1 ? 0 : r == 2 ? 1 : r == 4 ? 2 : 3) * NS + k];
          } else {
            w[r] = tw[r * ks];
          }
        } else {
          w[r] = cmul<float>(w[r & (r - 1)], w[r & -r]);
        }
      }
#pragma unroll
      for (int r = 1; r < R; ++r) v[q][r] = cmul<float>(v[q][r], mk<float>(w[r].x, DIR > 0 ? w[r].y : -w[r].y));
    }
    lnq[q] = line;
    dq[q] = (j - k) * R + k;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    dftR<float, DIR, R>(v[q]);
    if constexpr ((NS & 15) == 0) {
      CT* p = sm + lnq[q] * LP + dq[q] + (dq[q] >> 4);
#pragma unroll
      for (int r = 0; r < R; ++r) p[r * SWR] = v[q][r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) sm[sidx(lnq[q], LP, dq[q] + r * NS)] = v[q][r];
    }
  }
  __syncthreads();
}

template <int DIR, int LOGL, int LOGNS, int R0 = 0>
__device__ __forceinline__ void r16_stages_ct(C2<float>* sm, const C2<float>* __restrict__ tw) {
  if constexpr (LOGNS < LOGL) {
    stage_ct<DIR, 16, LOGL, LOGNS, R0>(sm, tw);
    r16_stages_ct<DIR, LOGL, LOGNS + 4, R0>(sm, tw);
  }
}

template <int DIR, int LOGL>
__device__ __forceinline__ void fft_tile_ct(C2<float>* sm, const C2<float>* __restrict__ tw) {
  constexpr int REM = LOGL & 3;
  if constexpr (REM == 1) stage_ct<DIR, 2, LOGL, 0>(sm, tw);
  if constexpr (REM == 2) stage_ct<DIR, 4, LOGL, 0>(sm, tw);
  if constexpr (REM == 3) stage_ct<DIR, 8, LOGL, 0>(sm, tw);
  r16_stages_ct<DIR, LOGL, REM>(sm, tw);
}

// Epilogue element of the i-th (thread, step) slot of a transposed tile write:
// row k of line c of a tile of C = 2^LOGC lines.  Each half-warp takes C lines
// x 16/C rows spaced C apart, so its reads of the padded tile (c LP + k + k/16,
// LP = 1 mod 16) hit 16 distinct bank pairs, while every warp still writes
// whole C-element row segments; slot tid + 256 q keeps the thread's line c and
// takes row k0 + (256/C) q.
template <int LOGC>
__device__ __forceinline__ void epi_slot(int i, int& k, int& c) {
  constexpr int C = 1 << LOGC;
  if constexpr (C >= 16) {
    k = i >> LOGC;
    c = i & (C - 1);
  } else {
    const int hw = i >> 4, l16 = i & 15;
    c = l16 & (C - 1);
    k = 16 * (hw >> LOGC) + (hw & (C - 1)) + C * (l16 >> LOGC);
  }
}

// Inter-pass twiddles of a column tile (columns c0 + c, c < C):
// T[q][c] = e^{2 pi i (256/C)(c0 + c) q / N}, q < 16, filled by the CTA (the
// lines of a half-warp read consecutive entries); the thread with line c and
// first row k0 multiplies B = e^{2 pi i (c0 + c) k0 / N} by T[q][c] for row
// k0 + (256/C) q.  Two rounded factors and one product, as
// with a two-level table, but only 16 C + 256 sines and cosines per tile and no
// global loads.
template <int LOGC>
__device__ __forceinline__ void tw_tile_fill(C2<float>* T, int c0, float two_over_n) {
  constexpr int C = 1 << LOGC;
  for (int j = threadIdx.x; j < 16 * C; j += FFT_THREADS) {
    const int q = j >> LOGC, c = j & (C - 1);
    T[j] = tw_pow2_f32((int64_t)(256 / C) * (c0 + c) * q, two_over_n);
  }
}

template <int DIR, int LOGL1>
__global__ void __launch_bounds__(FFT_THREADS, 4)
    k_fft32_cols(C2<float>* __restrict__ data, int64_t N, int L2, const C2<float>* __restrict__ tw4096,
                 const C2<float>* __restrict__ thi, const C2<float>* __restrict__ tlo, VecMap vm) {
  using CT = C2<float>;
  constexpr int L1 = 1 << LOGL1, LOGC = 12 - LOGL1, C = 1 << LOGC, LP = line_pitch_ct(L1);
  constexpr int PER = FFT_TILE / FFT_THREADS;
  __shared__ CT sm[C * LP];
  __shared__ CT tws[16 * C];
  const int c0 = blockIdx.x * C;
  CT* g = data + vec_of(vm, blockIdx.y) * N;
#pragma unroll
  for (int q0 = 0; q0 < PER; q0 += 8) {
    CT r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = threadIdx.x + (q0 + q) * FFT_THREADS;
      r[q] = g[(int64_t)(i >> LOGC) * L2 + c0 + (i & (C - 1))];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = threadIdx.x + (q0 + q) * FFT_THREADS;
      sm[sidx(i & (C - 1), LP, i >> LOGC)] = r[q];
    }
  }
  const float ton = 2.0f / (float)N;
  tw_tile_fill<LOGC>(tws, c0, ton);
  __syncthreads();
  fft_tile_ct<DIR, LOGL1>(sm, tw4096);
  int k0, c;
  epi_slot<LOGC>(threadIdx.x, k0, c);
  const CT B = tw_pow2_f32((int64_t)(c0 + c) * k0, ton);
#pragma unroll 4
  for (int q = 0; q < PER; ++q) {
    const int k1 = k0 + (256 / C) * q;
    const CT w = cmul<float>(B, tws[q * C + c]);
    const CT val = cmul<float>(sm[sidx(c, LP, k1)], mk<float>(w.x, DIR > 0 ? w.y : -w.y));
    g[(int64_t)k1 * L2 + c0 + c] = val;
  }
}

template <int DIR, int LOGL2>
__global__ void __launch_bounds__(FFT_THREADS, 4)
    k_fft32_rows(const C2<float>* __restrict__ in, C2<float>* __restrict__ out, int64_t N, int L1,
                 const C2<float>* __restrict__ tw4096, VecMap vm) {
  using CT = C2<float>;
  constexpr int L2 = 1 << LOGL2, LOGC2 = 12 - LOGL2, C2n = 1 << LOGC2, LP = line_pitch_ct(L2);
  constexpr int PER = FFT_TILE / FFT_THREADS;
  __shared__ CT sm[C2n * LP];
  const int r0 = blockIdx.x * C2n;
  const int64_t v = vec_of(vm, blockIdx.y);
  const CT* g = in + v * N + (int64_t)r0 * L2;
  CT* o = out + v * N;
#pragma unroll
  for (int q0 = 0; q0 < PER; q0 += 8) {
    CT r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = g[threadIdx.x + (q0 + q) * FFT_THREADS];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int i = threadIdx.x + (q0 + q) * FFT_THREADS;
      sm[sidx(i >> LOGL2, LP, i & (L2 - 1))] = r[q];
    }
  }
  __syncthreads();
  fft_tile_ct<DIR, LOGL2>(sm, tw4096);
#pragma unroll 4
  for (int q = 0; q < PER; ++q) {
    int k2, line;
    epi_slot<LOGC2>(threadIdx.x + q * FFT_THREADS, k2, line);
    o[(int64_t)(r0 + line) + (int64_t)L1 * k2] = sm[sidx(line, LP, k2)];
  }
}

// launch the FP32 compile-time pass for log2 L in [6, 12]; false if none applies
template <int DIR>
static bool launch_fft32_cols(int logL1, dim3 grid, cudaStream_t s, C2<float>* a, int64_t N, int L2,
                              const C2<float>* tw, const C2<float>* thi, const C2<float>* tlo, VecMap vm) {
  switch (logL1) {
#define GBDLT_C32(LG) \
  case LG:            \
    k_fft32_cols<DIR, LG><<<grid, FFT_THREADS, 0, s>>>(a, N, L2, tw, thi, tlo, vm); \
    return true;
    GBDLT_C32(6) GBDLT_C32(7) GBDLT_C32(8) GBDLT_C32(9) GBDLT_C32(10) GBDLT_C32(11) GBDLT_C32(12)
#undef GBDLT_C32
  }
  return false;
}
template <int DIR>
static bool launch_fft32_rows(int logL2, dim3 grid, cudaStream_t s, const C2<float>* a, C2<float>* b, int64_t N,
                              int L1, const C2<float>* tw, VecMap vm) {
  switch (logL2) {
#define GBDLT_R32(LG) \
  case LG:            \
    k_fft32_rows<DIR, LG><<<grid, FFT_THREADS, 0, s>>>(a, b, N, L1, tw, vm); \
    return true;
    GBDLT_R32(6) GBDLT_R32(7) GBDLT_R32(8) GBDLT_R32(9) GBDLT_R32(10) GBDLT_R32(11) GBDLT_R32(12)
#undef GBDLT_R32
  }
  return false;
}

// ---------------------------------------------------------------- FP32 passes staged by TMA
// The compile-time FP32 passes above load each tile with per-thread global loads
// before the first butterfly and store it after the last, so while a CTA
// computes it has nothing in flight, and the 3-4 CTAs an SM holds leave the
// memory system idle much of the time.  The passes below are persistent (a grid
// of 3 CTAs per SM stepping over the tiles) and move each tile with the tensor
// memory accelerator into a staging buffer of its own:
//   * column pass: a 3-D tensor map over the buffer viewed as
//     [vector][row n1 < L1][2 L2 floats]; one tile (C = 4096/L1 adjacent
//     columns of one vector) is L1/256 boxes of 256 rows x 2C floats
//     (cp.async.bulk.tensor), landing unpadded as [n1][c];
//   * row pass: a tile is C2 = 4096/L2 whole rows, one contiguous 32 KB run,
//     moved by one bulk copy (cp.async.bulk).
// The first Stockham stage (no twiddles) reads the staging buffer and writes the
// padded work tile of the generic kernels; once every thread has passed it, one
// thread issues the copy of the CTA's next tile into the staging buffer, so that
// copy runs under the remaining stages, the inter-pass twiddle and the stores of
// the current tile.  In the column pass the first stage takes the column index
// as the fastest-varying thread index: it then reads the unpadded [n1][c] tile
// and writes the padded one without bank conflicts for every line length of
// 2^13 <= N <= 2^23 (a model of the 16 bank pairs of 8-byte accesses).
// Completion is an mbarrier with a transaction count.  Every wait is bounded
// (about 2 s of SM clock): a copy that has not landed by then sets bit 2 of the
// plan's status word (gbdlt_plan_sync reports a CUDA error) and the CTA returns.
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this CTA's earlier generic-proxy accesses of shared memory before later
// async-proxy (TMA) accesses
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// SM cycles a staged pass waits for a tile copy before it gives up (about 2 s)
constexpr long long kWaitCycles = 1ll << 32;
// non-blocking test of phase `parity` (try_wait may suspend the thread for a
// while before it answers)
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// true once phase `parity` of the barrier has completed; false after `limit` SM
// cycles without completion (limit 0: unless it has completed already)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_test_wait(bar, parity)) return true;
  if (limit <= 0) return false;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}
// A wait that ran out: record it in the plan status (bit 2) and wait once more,
// with the full limit, for the CTA's own copy in flight before the CTA returns,
// so that no copy lands in shared memory the CTA no longer owns.
__device__ __forceinline__ void give_up(uint64_t* bar, uint32_t parity, int* status) {
  if (threadIdx.x == 0) {
    atomicOr(status, 2);
    mbar_wait(bar, parity, kWaitCycles);
  }
  __syncthreads();
}
__device__ __forceinline__ void load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

}  // namespace tma

// First Stockham stage (radix R, sub-transform length 1, no twiddles) of `lines`
// lines of length L = 2^LOGL held unpadded in the staging buffer S, written to
// the padded work tile W.  COLS: S is [i][line] (column-pass tile) and the line
// index varies fastest over the threads; otherwise S is [line][i].
template <int DIR, int R, int LOGL, bool COLS>
__device__ __forceinline__ void stage_first_ct(const C2<float>* __restrict__ S, C2<float>* __restrict__ W) {
  using CT = C2<float>;
  constexpr int L = 1 << LOGL;
  constexpr int LOGR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
  constexpr int LR = L / R, LOGLR = LOGL - LOGR;
  constexpr int LOGC = 12 - LOGL, C = 1 << LOGC;
  constexpr int LP = line_pitch_ct(L);
  constexpr int PER = FFT_TILE / R / FFT_THREADS;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int b = threadIdx.x + q * FFT_THREADS;
    const int line = COLS ? (b & (C - 1)) : (b >> LOGLR);
    const int j = COLS ? (b >> LOGC) : (b & (LR - 1));
    CT v[R];
    if constexpr (COLS) {
      const CT* p = S + j * C + line;
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = p[r * LR * C];
    } else {
      const CT* p = S + line * L + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = p[r * LR];
    }
    dftR<float, DIR, R>(v);
    // outputs j R + r, r < R: one base plus immediate offsets (R divides 16)
    CT* o = W + line * LP + j * R + ((j * R) >> 4);
#pragma unroll
    for (int r = 0; r < R; ++r) o[r] = v[r];
  }
  __syncthreads();
}

// tw: the shared-memory twiddle rows of tw_fill
template <int DIR, int LOGL, bool COLS>
__device__ __forceinline__ void fft_tile_staged(const C2<float>* S, C2<float>* W, const C2<float>* __restrict__ tw,
                                                uint64_t* bar, bool issue_next, const void* next_src,
                                                const CUtensorMap* map, int nx, int ny, int nz) {
  constexpr int REM = LOGL & 3;
  constexpr int R0 = REM == 1 ? 2 : REM == 2 ? 4 : REM == 3 ? 8 : 16;
  stage_first_ct<DIR, R0, LOGL, COLS>(S, W);
  // every thread has read S: refill it with the CTA's next tile
  if (issue_next && threadIdx.x == 0) {
    tma::fence_proxy_async();
    tma::mbar_expect_tx(bar, FFT_TILE * sizeof(C2<float>));
    if constexpr (COLS) {
      constexpr int L = 1 << LOGL, BOXR = L < 256 ? L : 256;
#pragma unroll 1
      for (int r = 0; r < L; r += BOXR) tma::load_3d((char*)S + (size_t)r * (FFT_TILE / L) * sizeof(C2<float>), map,
                                                     nx, ny + r, nz, bar);
    } else {
      tma::load_1d((void*)S, next_src, FFT_TILE * sizeof(C2<float>), bar);
    }
  }
  r16_stages_ct<DIR, LOGL, (REM == 0 ? 4 : REM), (REM == 0 ? 16 : (1 << REM))>(W, tw);
}

// Shared-memory twiddles of the radix-16 stages of a line of length L = 2^LOGL
// (first stage radix R0, untwiddled): stage NS = R0 16^s (NS < L) holds four
// rows [b][k], k < NS, with tw4096[2^b k 4096 / (16 NS)] = e^{2 pi i 2^b k /
// (16 NS)}, the same rounded values the global table gives, so the staged passes
// stay bitwise equal to the others.  Entries: 4 (L - R0) / 15.
template <int LOGL>
__host__ __device__ constexpr int tw_rows_r0() {
  return (LOGL & 3) == 0 ? 16 : 1 << (LOGL & 3);
}
template <int LOGL>
__host__ __device__ constexpr int tw_rows_len() {
  return 4 * ((1 << LOGL) - tw_rows_r0<LOGL>()) / 15;
}
template <int LOGL>
__device__ __forceinline__ void tw_fill(C2<float>* T, const C2<float>* __restrict__ tw4096) {
  constexpr int R0 = tw_rows_r0<LOGL>(), L = 1 << LOGL;
  for (int e = threadIdx.x; e < tw_rows_len<LOGL>(); e += FFT_THREADS) {
    // stage of entry e: offsets 4 (NS - R0) / 15 for NS = R0, 16 R0, ...
    int NS = R0;
    while (NS * 16 < L && e >= 4 * (NS * 16 - R0) / 15) NS *= 16;
    const int o = e - 4 * (NS - R0) / 15;
    const int b = o / NS, k = o % NS;
    T[e] = tw4096[(1 << b) * k * (FFT_TILE / (16 * NS))];
  }
}

template <int DIR, int LOGL1>
__global__ void __launch_bounds__(FFT_THREADS, 3)
    k_fft32_cols_tma(const __grid_constant__ CUtensorMap map, C2<float>* __restrict__ data, int64_t N, int L2,
                     const C2<float>* __restrict__ tw4096, const C2<float>* __restrict__ thi,
                     const C2<float>* __restrict__ tlo, VecMap vm, int64_t ntiles, int* __restrict__ status,
                     long long wait_limit) {
  using CT = C2<float>;
  constexpr int L1 = 1 << LOGL1, LOGC = 12 - LOGL1, C = 1 << LOGC, LP = line_pitch_ct(L1);
  constexpr int PER = FFT_TILE / FFT_THREADS;
  constexpr int BOXR = L1 < 256 ? L1 : 256;
  extern __shared__ __align__(1024) unsigned char smraw[];
  CT* S = reinterpret_cast<CT*>(smraw);
  CT* W = S + FFT_TILE;
  CT* T = W + C * LP;
  CT* tws = T + tw_rows_len<LOGL1>();
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + 16 * C);
  const float ton = 2.0f / (float)N;
  const int nblk = L2 / C;
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  if (threadIdx.x == 0) {
    tma::mbar_init(bar, 1);
    tma::fence_mbar_init();
  }
  tw_fill<LOGL1>(T, tw4096);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t v = vec_of(vm, t / nblk);
    const int c0 = (int)(t % nblk) * C;
    tma::mbar_expect_tx(bar, FFT_TILE * sizeof(CT));
#pragma unroll 1
    for (int r = 0; r < L1; r += BOXR)
      tma::load_3d((char*)S + (size_t)r * C * sizeof(CT), &map, 2 * c0, r, (int)v, bar);
  }
  uint32_t phase = 0;
  for (; t < ntiles; t += gridDim.x) {
    const bool ok = tma::mbar_wait(bar, phase, wait_limit);
    if (__syncthreads_or(!ok)) {
      tma::give_up(bar, phase, status);
      return;
    }
    phase ^= 1;
    const int64_t v = vec_of(vm, t / nblk);
    const int c0 = (int)(t % nblk) * C;
    const int64_t tn = t + gridDim.x;
    const bool more = tn < ntiles;
    tw_tile_fill<LOGC>(tws, c0, ton);  // read after the stages' barriers
    fft_tile_staged<DIR, LOGL1, true>(S, W, T, bar, more, nullptr, &map,
                                      more ? 2 * (int)(tn % nblk) * C : 0, 0, more ? (int)vec_of(vm, tn / nblk) : 0);
    CT* g = data + v * N;
    int k0, c;
    epi_slot<LOGC>(threadIdx.x, k0, c);
    const CT B = tw_pow2_f32((int64_t)(c0 + c) * k0, ton);
#pragma unroll 4
    for (int q = 0; q < PER; ++q) {
      const int k1 = k0 + (256 / C) * q;
      const CT w = cmul<float>(B, tws[q * C + c]);
      const CT val = cmul<float>(W[sidx(c, LP, k1)], mk<float>(w.x, DIR > 0 ? w.y : -w.y));
      g[(int64_t)k1 * L2 + c0 + c] = val;
    }
    __syncthreads();  // W and the tile twiddles are rewritten for the next tile
  }
}

template <int DIR, int LOGL2>
__global__ void __launch_bounds__(FFT_THREADS, 3)
    k_fft32_rows_tma(const C2<float>* __restrict__ in, C2<float>* __restrict__ out, int64_t N, int L1,
                     const C2<float>* __restrict__ tw4096, VecMap vm, int64_t ntiles, int* __restrict__ status,
                     long long wait_limit) {
  using CT = C2<float>;
  constexpr int L2 = 1 << LOGL2, LOGC2 = 12 - LOGL2, C2n = 1 << LOGC2, LP = line_pitch_ct(L2);
  constexpr int PER = FFT_TILE / FFT_THREADS;
  extern __shared__ __align__(1024) unsigned char smraw[];
  CT* S = reinterpret_cast<CT*>(smraw);
  CT* W = S + FFT_TILE;
  CT* T = W + C2n * LP;
  uint64_t* bar = reinterpret_cast<uint64_t*>(T + tw_rows_len<LOGL2>());
  const int nblk = L1 / C2n;
  int64_t t = blockIdx.x;
  if (t >= ntiles) return;
  if (threadIdx.x == 0) {
    tma::mbar_init(bar, 1);
    tma::fence_mbar_init();
  }
  tw_fill<LOGL2>(T, tw4096);
  __syncthreads();
  auto src_of = [&](int64_t tt) {
    return in + vec_of(vm, tt / nblk) * N + (int64_t)(tt % nblk) * C2n * L2;
  };
  if (threadIdx.x == 0) {
    tma::mbar_expect_tx(bar, FFT_TILE * sizeof(CT));
    tma::load_1d(S, src_of(t), FFT_TILE * sizeof(CT), bar);
  }
  uint32_t phase = 0;
  for (; t < ntiles; t += gridDim.x) {
    const bool ok = tma::mbar_wait(bar, phase, wait_limit);
    if (__syncthreads_or(!ok)) {
      tma::give_up(bar, phase, status);
      return;
    }
    phase ^= 1;
    const int64_t v = vec_of(vm, t / nblk);
    const int r0 = (int)(t % nblk) * C2n;
    const int64_t tn = t + gridDim.x;
    const bool more = tn < ntiles;
    fft_tile_staged<DIR, LOGL2, false>(S, W, T, bar, more, more ? (const void*)src_of(tn) : nullptr, nullptr,
                                       0, 0, 0);
    CT* o = out + v * N;
#pragma unroll 4
    for (int q = 0; q < PER; ++q) {
      int k2, line;
      epi_slot<LOGC2>(threadIdx.x + q * FFT_THREADS, k2, line);
      o[(int64_t)(r0 + line) + (int64_t)L1 * k2] = W[sidx(line, LP, k2)];
    }
    __syncthreads();
  }
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
// the driver's tensor-map encoder, looked up once (null if the driver has none)
EncodeTiled encode_tiled() {
  static EncodeTiled fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiled) nullptr;
    }
    return (EncodeTiled)f;
  }();
  return fn;
}

int sm_count() {
  static int count[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 148;
  if (!count[dev]) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) {
      cudaGetLastError();
      c = 148;
    }
    count[dev] = c;
  }
  return count[dev];
}

// raise a staged kernel's dynamic shared-memory limit once (before the first
// launch of any call, which runs uncaptured)
std::mutex g_smem_mu;
std::vector<const void*> g_smem_set;
template <typename K>
bool set_smem(K kernel, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_smem_mu);
  const void* key = (const void*)kernel;
  for (const void* k : g_smem_set)
    if (k == key) return true;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  g_smem_set.push_back(key);
  return true;
}
}  // namespace

// dynamic shared memory of a staged FP32 pass over lines of length L: staging
// tile, padded work tile, twiddle rows (at most L/2 entries), the column pass's
// tile twiddles (16 C entries), mbarrier
constexpr size_t tma_smem_bytes(int L) {
  return (size_t)(FFT_TILE + (FFT_TILE / L) * line_pitch_ct(L) + L / 2 + 16 * (FFT_TILE / L)) * sizeof(C2<float>) +
         16;
}

// The staged FP32 column pass for log2 L1 in [7, 11] (2 <= C <= 32, so a box row
// is 16..256 bytes); false (nothing launched) where it does not apply.
template <int DIR>
static bool launch_fft32_cols_tma(int logL1, Plan& P, C2<float>* a, int64_t N, int L2, const C2<float>* tw,
                                  const C2<float>* thi, const C2<float>* tlo, VecMap vm, int64_t nv) {
  if (logL1 < 7 || logL1 > 11 || P.no_tma) return false;
  EncodeTiled enc = encode_tiled();
  if (!enc) return false;
  const int L1 = 1 << logL1, C = FFT_TILE / L1;
  const int64_t vmax = vec_of_host(vm, nv - 1);
  CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * L2, (cuuint64_t)L1, (cuuint64_t)(vmax + 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)L2 * sizeof(C2<float>), (cuuint64_t)N * sizeof(C2<float>)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * C), (cuuint32_t)(L1 < 256 ? L1 : 256), 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)a, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return false;
  const int64_t ntiles = nv * (L2 / C);
  const int64_t grid = std::min<int64_t>(ntiles, 3 * (int64_t)sm_count());
  const size_t smem = tma_smem_bytes(L1);
  switch (logL1) {
#define GBDLT_C32T(LG)                                                                                        \
  case LG:                                                                                                    \
    if (!set_smem(k_fft32_cols_tma<DIR, LG>, smem)) return false;                                             \
    k_fft32_cols_tma<DIR, LG><<<(unsigned)grid, FFT_THREADS, smem, P.stream>>>(map, a, N, L2, tw, thi, tlo, vm, \
                                                                               ntiles, P.status, P.tma_wait); \
    return true;
    GBDLT_C32T(7) GBDLT_C32T(8) GBDLT_C32T(9) GBDLT_C32T(10) GBDLT_C32T(11)
#undef GBDLT_C32T
  }
  return false;
}

// The staged FP32 row pass for log2 L2 in [6, 10]; at L2 = 2048 (N = 2^22,
// 2^23), where a tile is two rows and its stores 16-byte pieces, the staged pass
// measured slower than the per-thread-load pass (1.18 against 0.81 ms for the
// FP32 form's six launches at 2^22) and is not used.
template <int DIR>
static bool launch_fft32_rows_tma(int logL2, Plan& P, const C2<float>* a, C2<float>* b, int64_t N, int L1,
                                  const C2<float>* tw, VecMap vm, int64_t nv) {
  if (logL2 < 6 || logL2 > 10 || P.no_tma) return false;
  const int L2 = 1 << logL2, C2n = FFT_TILE / L2;
  const int64_t ntiles = nv * (L1 / C2n);
  const int64_t grid = std::min<int64_t>(ntiles, 3 * (int64_t)sm_count());
  const size_t smem = tma_smem_bytes(L2);
  switch (logL2) {
#define GBDLT_R32T(LG)                                                                                              \
  case LG:                                                                                                          \
    if (!set_smem(k_fft32_rows_tma<DIR, LG>, smem)) return false;                                                   \
    k_fft32_rows_tma<DIR, LG><<<(unsigned)grid, FFT_THREADS, smem, P.stream>>>(a, b, N, L1, tw, vm, ntiles, P.status, \
                                                                               P.tma_wait);                    \
    return true;
    GBDLT_R32T(6) GBDLT_R32T(7) GBDLT_R32T(8) GBDLT_R32T(9) GBDLT_R32T(10)
#undef GBDLT_R32T
  }
  return false;
}

template <typename T, int DIR>
static void* four_step(Plan& P, void* a, void* b, int64_t nb, int64_t per_item, int64_t npruned, int R,
                       int mode);

// the tile kernels use more than 48 KB of dynamic shared memory: raise their
// limit once per (T, DIR), before the first launch from any entry path
template <typename T, int DIR>
static void fft_attrs() {
  static bool done = false;
  if (done) return;
  const int smax = (int)(FFT_SMEM_ELEMS * sizeof(C2<T>));
  cudaFuncSetAttribute(k_fft_single<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  cudaFuncSetAttribute(k_fft_cols<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  cudaFuncSetAttribute(k_fft_rows<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  done = true;
}

template <typename T, int DIR>
static void* fft_dir(Plan& P, void* a, void* b, int64_t nvec) {
  using CT = C2<T>;
  const int64_t N = P.p.N;
  if (nvec <= 0 || N <= 1) return a;
  const TwT<T> tw = tw_tables(P, T());
  // cosine/tangent table of this direction (FP64 only)
  const double2* lfd = tw.lf ? tw.lf + (DIR > 0 ? 0 : 2 * 4096) : nullptr;
  fft_attrs<T, DIR>();
  if (N <= FFT_TILE) {
    int L = (int)N;
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    int lines = FFT_TILE / L;
    int64_t grid = (nvec + lines - 1) / lines;
    size_t sm = (size_t)lines * line_pitch(L) * sizeof(CT);
    k_fft_single<T, DIR><<<(unsigned)grid, FFT_THREADS, sm, P.stream>>>((CT*)a, L, lg, nvec, tw.t4096, lfd);
    launched(P, kname<T>("fft_single", "fft32_single", "fftff_single"), 5.0 * (double)N * lg * nvec, 2.0 * (double)nvec * N * sizeof(CT));
    return a;
  }
  return four_step<T, DIR>(P, a, b, nvec, 1, 0, 0, 0);
}

// Four-step FFT of nb items x per_item vectors; the first npruned vectors of
// every item are pruned to the windows of half-width R: their row pass (mode 1,
// forward, output windows) or column pass (mode 2, transposed, input windows)
// runs in the pruned kernel, all other passes in the full kernels.
template <typename T, int DIR>
static void* four_step(Plan& P, void* a, void* b, int64_t nb, int64_t per_item, int64_t npruned, int R,
                       int mode) {
  using CT = C2<T>;
  fft_attrs<T, DIR>();
  const int64_t N = P.p.N;
  const TwT<T> tw = tw_tables(P, T());
  const double2* lfd = tw.lf ? tw.lf + (DIR > 0 ? 0 : 2 * 4096) : nullptr;
  int p = 0;
  while ((1ll << p) < N) ++p;
  const int L1 = 1 << (p / 2);
  const int L2 = (int)(N / L1);
  const int C = FFT_TILE / L1;
  const int C2n = FFT_TILE / L2;
  const int lL1 = p / 2, lL2 = p - p / 2, lC = 12 - lL1, lC2 = 12 - lL2;
  if (mode == 0 || 2 * R > L1 || 2 * R > L2 || C > 64) npruned = 0;
  const int64_t nfull = per_item - npruned;
  const VecMap all{0, nb * per_item, nb * per_item};
  const VecMap pruned{0, npruned, per_item};
  const VecMap rest{npruned, nfull, per_item};
  const size_t smc = (size_t)C * line_pitch(L1) * sizeof(CT), smr = (size_t)C2n * line_pitch(L2) * sizeof(CT);
  // full column / row passes over a vector map: the FP32 compile-time kernels
  // where the line length has one, else the generic ones
  auto cols = [&](VecMap vm, int64_t nv) {
    const dim3 grid(L2 / C, (unsigned)nv);
    if constexpr (is_f32<T>) {
      if (launch_fft32_cols_tma<DIR>(lL1, P, (C2<float>*)a, N, L2, (const C2<float>*)tw.t4096,
                                     (const C2<float>*)tw.nhi, (const C2<float>*)tw.nlo, vm, nv))
        return;
      if (launch_fft32_cols<DIR>(lL1, grid, P.stream, (C2<float>*)a, N, L2, (const C2<float>*)tw.t4096,
                                 (const C2<float>*)tw.nhi, (const C2<float>*)tw.nlo, vm))
        return;
    }
    k_fft_cols<T, DIR><<<grid, FFT_THREADS, smc, P.stream>>>((CT*)a, N, L1, lL1, L2, C, lC, tw.t4096, tw.nhi,
                                                              tw.nlo, tw.full, lfd, vm);
  };
  auto rows = [&](VecMap vm, int64_t nv) {
    const dim3 grid(L1 / C2n, (unsigned)nv);
    if constexpr (is_f32<T>) {
      if (launch_fft32_rows_tma<DIR>(lL2, P, (const C2<float>*)a, (C2<float>*)b, N, L1, (const C2<float>*)tw.t4096,
                                     vm, nv))
        return;
      if (launch_fft32_rows<DIR>(lL2, grid, P.stream, (const C2<float>*)a, (C2<float>*)b, N, L1,
                                 (const C2<float>*)tw.t4096, vm))
        return;
    }
    k_fft_rows<T, DIR><<<grid, FFT_THREADS, smr, P.stream>>>((const CT*)a, (CT*)b, N, L1, L2, lL2, C2n, lC2,
                                                              tw.t4096, lfd, vm);
  };
  // column pass
  if (mode == 2 && npruned > 0) {
    k_fft_cols_pruned<T, DIR><<<dim3(L2 / C, (unsigned)(nb * npruned)), FFT_THREADS, 0, P.stream>>>(
        (CT*)a, N, L1, L2, R, C, lC, tw.nhi, tw.nlo, tw.full, pruned);
    launched(P, kname<T>("fft_cols_pruned", "fft32_cols_pruned", "fftff_cols_pruned"), 6.0 * (double)N * nb * npruned * (4.0 * R / L2),
             (double)nb * npruned * N * sizeof(CT));
    if (nfull > 0) {
      cols(rest, nb * nfull);
      launched(P, kname<T>("fft_cols", "fft32_cols", "fftff_cols"), (5.0 * lL1 + 6.0) * (double)N * nb * nfull, 2.0 * (double)nb * nfull * N * sizeof(CT));
    }
  } else {
    cols(all, nb * per_item);
    launched(P, kname<T>("fft_cols", "fft32_cols", "fftff_cols"), (5.0 * lL1 + 6.0) * (double)N * nb * per_item,
             2.0 * (double)nb * per_item * N * sizeof(CT));
  }
  // row pass
  if (mode == 1 && npruned > 0) {
    k_fft_rows_pruned<T, DIR><<<dim3((2 * R + 7) / 8, (unsigned)(nb * npruned)), FFT_THREADS, 0, P.stream>>>(
        (const CT*)a, (CT*)b, N, L1, L2, R, tw.t4096, pruned);
    launched(P, kname<T>("fft_rows_pruned", "fft32_rows_pruned", "fftff_rows_pruned"), 6.0 * 2.0 * R * L2 * (double)nb * npruned,
             (double)nb * npruned * 2.0 * R * L2 * sizeof(CT));
    if (nfull > 0) {
      rows(rest, nb * nfull);
      launched(P, kname<T>("fft_rows", "fft32_rows", "fftff_rows"), 5.0 * lL2 * (double)N * nb * nfull, 2.0 * (double)nb * nfull * N * sizeof(CT));
    }
  } else {
    rows(all, nb * per_item);
    launched(P, kname<T>("fft_rows", "fft32_rows", "fftff_rows"), 5.0 * lL2 * (double)N * nb * per_item, 2.0 * (double)nb * per_item * N * sizeof(CT));
  }
  return b;
}

// The FP64 and float-float vectors of one stage (both of length N > 4096, the
// four-step sizes) through the mixed passes; results in b64 and bff.
template <int DIR>
static void fft_mix_dir(Plan& P, void* a64, void* b64, int64_t nv64, void* aff, void* bff, int64_t nvff) {
  static bool attr = false;
  const int smax = (int)(FFT_SMEM_ELEMS * sizeof(C2<double>));
  if (!attr) {
    cudaFuncSetAttribute(k_fft_cols_mix<DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    cudaFuncSetAttribute(k_fft_rows_mix<DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
    attr = true;
  }
  const int64_t N = P.p.N;
  int p = 0;
  while ((1ll << p) < N) ++p;
  const int L1 = 1 << (p / 2);
  const int L2 = (int)(N / L1);
  const int C = FFT_TILE / L1;
  const int C2n = FFT_TILE / L2;
  const int lL1 = p / 2, lL2 = p - p / 2, lC = 12 - lL1, lC2 = 12 - lL2;
  const TwT<double> tw = tw_tables(P, double());
  const double2* lfd = tw.lf ? tw.lf + (DIR > 0 ? 0 : 2 * 4096) : nullptr;
  MixArgs M;
  M.a64 = (C2<double>*)a64;
  M.b64 = (C2<double>*)b64;
  M.aff = (ffc*)aff;
  M.bff = (ffc*)bff;
  M.vm64 = VecMap{0, std::max<int64_t>(nv64, 1), std::max<int64_t>(nv64, 1)};
  M.vmff = VecMap{0, std::max<int64_t>(nvff, 1), std::max<int64_t>(nvff, 1)};
  const size_t smc = (size_t)C * line_pitch(L1) * sizeof(C2<double>);
  const size_t smr = (size_t)C2n * line_pitch(L2) * sizeof(C2<double>);
  const int nxc = L2 / C, nxr = L1 / C2n;
  M.n64 = (int64_t)nxc * nv64;
  M.nff = (int64_t)nxc * nvff;
  k_fft_cols_mix<DIR><<<(unsigned)(M.n64 + M.nff), FFT_THREADS, smc, P.stream>>>(
      M, N, L1, lL1, L2, C, lC, nxc, tw.t4096, tw.full, lfd, P.tw4096_ff, P.twfull_ff);
  launched(P, "fftmix_cols", (5.0 * lL1 + 6.0) * (double)N * (double)(nv64 + nvff),
           2.0 * (double)(nv64 + nvff) * N * 16.0);
  M.n64 = (int64_t)nxr * nv64;
  M.nff = (int64_t)nxr * nvff;
  k_fft_rows_mix<DIR><<<(unsigned)(M.n64 + M.nff), FFT_THREADS, smr, P.stream>>>(M, N, L1, L2, lL2, C2n, lC2,
                                                                                  nxr, tw.t4096, lfd,
                                                                                  P.tw4096_ff);
  launched(P, "fftmix_rows", 5.0 * lL2 * (double)N * (double)(nv64 + nvff), 2.0 * (double)(nv64 + nvff) * N * 16.0);
}

void launch_fft_mix(Plan& P, void* a64, void* b64, int64_t nv64, void* aff, void* bff, int64_t nvff, int dir) {
  if (dir > 0)
    fft_mix_dir<1>(P, a64, b64, nv64, aff, bff, nvff);
  else
    fft_mix_dir<-1>(P, a64, b64, nv64, aff, bff, nvff);
}

template <typename T>
void* launch_fft(Plan& P, void* a, void* b, int64_t nvec, int dir) {
  return dir > 0 ? fft_dir<T, 1>(P, a, b, nvec) : fft_dir<T, -1>(P, a, b, nvec);
}

template <typename T>
void* launch_fft_bands(Plan& P, void* a, void* b, int64_t nb, int dir, int transposed, int terms) {
  const int64_t KM = (int64_t)P.p.K * terms;
  if (P.p.N <= FFT_TILE || P.prune_bands == 0) return launch_fft<T>(P, a, b, nb * KM, dir);
  const int64_t np = (int64_t)P.prune_bands * terms;
  const int mode = transposed ? 2 : 1;
  return dir > 0 ? four_step<T, 1>(P, a, b, nb, KM, np, P.prune_R, mode)
                 : four_step<T, -1>(P, a, b, nb, KM, np, P.prune_R, mode);
}

template void* launch_fft<double>(Plan&, void*, void*, int64_t, int);
template void* launch_fft_bands<double>(Plan&, void*, void*, int64_t, int, int, int);
template void* launch_fft_bands<float>(Plan&, void*, void*, int64_t, int, int, int);
template void* launch_fft_bands<ffd>(Plan&, void*, void*, int64_t, int, int, int);

namespace {
// cosine/tangent table for both directions: entry e of direction d holds the
// form of e^{i a}, a = (d ? -1 : +1) 2 pi e / 4096
__global__ void k_lf_init(double2* __restrict__ tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * 4096) return;
  const int d = i >> 12, e = i & 4095;
  double s, c;
  sincospi(2.0 * (double)e / 4096.0, &s, &c);
  if (d) s = -s;
  double sx, sy, t, sw;
  if (fabs(c) >= fabs(s)) {
    sx = c;
    sy = c;
    t = s / c;
    sw = 0.0;
  } else {
    sx = -s;
    sy = s;
    t = c / s;
    sw = 1.0;
  }
  tab[2 * i] = make_double2(sx, sy);
  tab[2 * i + 1] = make_double2(t, sw);
}
}  // namespace

namespace {
// float-float copies of FP64 twiddles: hi = fl(v), lo = fl(v - hi)
__global__ void k_tw_to_ff(const double2* __restrict__ in, ffc* __restrict__ out, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double2 v = in[i];
  const float xh = __double2float_rn(v.x), yh = __double2float_rn(v.y);
  ffc w;
  w.x = ffd(xh, __double2float_rn(v.x - (double)xh));
  w.y = ffd(yh, __double2float_rn(v.y - (double)yh));
  out[i] = w;
}
}  // namespace

int launch_fft_tables_init(Plan& P) {
  if (P.lf_tab) {
    k_lf_init<<<32, 256, 0, P.stream>>>(P.lf_tab);
    count_launch();
  }
  if (P.tw4096_ff) {
    k_tw_to_ff<<<16, 256, 0, P.stream>>>(P.tw4096, P.tw4096_ff, 4096);
    count_launch();
  }
  if (P.twfull_ff && P.twfull) {
    k_tw_to_ff<<<(unsigned)((P.p.N + 255) / 256), 256, 0, P.stream>>>(P.twfull, P.twfull_ff, P.p.N);
    count_launch();
  }
  return check_launch();
}
template void* launch_fft<float>(Plan&, void*, void*, int64_t, int);
template void* launch_fft<ffd>(Plan&, void*, void*, int64_t, int);

}  // namespace gbdlt
