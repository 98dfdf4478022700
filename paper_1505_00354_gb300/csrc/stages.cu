// Pre- and post-processing kernels around the FFT engine.
//
// Grid: theta_k = (k+1/2) pi / N, the Chebyshev points of the first kind (Eq. 5).
// Every DCT/DST the method needs (Eq. 13 and its transpose, Sec. 4 item 2) is
// one complex FFT of length N through one of three reductions:
//
//  FCS  (forward, one real input a):  Z_k = sum_n a_n e^{i n theta_k}.
//       u_n = a_n e^{i pi n/(2N)},  y = FFT+(u),  Z_{2m} = y_m,
//       Z_{2m+1} = conj(y_{N-1-m}).  Re Z is the DCT-III of Sec. 2.3, Im Z the DST-III.
//  F2   (forward pair, X of a and Y of b):  U_n = e^{i pi n/(2N)} [(a_n + b_n) - i(a_{N-n} - b_{N-n})],
//       U_0 = 2 a_0, y = FFT+(U);  X_a(2m) = Re y_m / 2, X_a(2m+1) = Re y_{N-1-m} / 2,
//       Y_b(k) = (-1)^k Im y_{m'} / 2 at the same index (a_N = b_N = 0).
//  T2   (transposed pair, DCT-II of a and DST-II of b):  with h_k = (-1)^k b_k,
//       v_{k'} = a_{2k'} + i h_{2k'},  v_{N-1-k'} = a_{2k'+1} + i h_{2k'+1},  F = FFT-(v);
//       U_n = Re[e^{-i pi n/(2N)} (F_n + conj F_{N-n})/2],
//       V_n = Re[e^{-i pi (N-n)/(2N)} (F_{N-n} - conj F_n)/(2i)]  (V_0 = 0).
//
// Stage kernels (one launch each; thread per output element):
//  l2c_pro / l2c_epi   asymptotic part of leg2cheb (Sec. 3, expansion of
//                      P_n(cos theta)): per band s and term m the FCS of
//                      a^{(m)}_n = C_n h_{m,n} c_n [n >= ns], combined as
//                      v_k += sum_m Re[e^{i(m+1/2)(theta_k - pi/2)} Z^{(s,m)}_k] / (2 sin theta_k)^{m+1/2}
//  a4_pro / a4_epi     values on the cheb1 grid -> Chebyshev coefficients:
//                      chat_j = (2/N) sum_k v_k cos(j theta_k), halved at j = 0
//  tay_pro / tay_epi   Taylor NDCT, Eq. (13): f_k = [v_k] + sum_l Re[(i t_k)^l/l! Z_l(k)],
//                      Z_l = FCS((n/N)^l chat), t_k = N dtheta_k; terms paired (F2)
//  tayt_pro / tayt_epi transposed Taylor sum (Sec. 4 item 2), pairs through T2
//  l2ct_pro / l2ct_epi transposed asymptotic part (Sec. 4 item 3)
#include <algorithm>

#include "gbdlt_internal.cuh"

namespace gbdlt {

namespace {

struct BandArgs {
  int K;
  int64_t ns[GBDLT_MAX_BANDS];
  int64_t ka[GBDLT_MAX_BANDS];
  int64_t kb[GBDLT_MAX_BANDS];
};

BandArgs band_args(const Plan& P) {
  BandArgs b{};
  b.K = P.p.K;
  for (int s = 0; s < P.p.K; ++s) {
    b.ns[s] = P.p.bands[s].ns;
    b.ka[s] = P.p.bands[s].ka;
    b.kb[s] = P.p.bands[s].kb;
  }
  return b;
}

template <typename T>
struct TwArgs {
  const C2<T>* hi;
  const C2<T>* lo;
};

// e^{2 pi i e / B} from the two-level table, multiplied in precision T
template <typename T>
__device__ __forceinline__ C2<T> twid(TwArgs<T> t, int64_t e) {
  return cmul<T>(t.hi[e >> 12], t.lo[e & 4095]);
}

template <typename T>
TwArgs<T> tw4n_args(const Plan& P) {
  const TwT<T> t = tw_tables(P, T());
  return TwArgs<T>{t.fhi, t.flo};
}

__device__ __forceinline__ void sincospi_t(double a, double* s, double* c) { sincospi(a, s, c); }
__device__ __forceinline__ void sincospi_t(float a, float* s, float* c) { sincospif(a, s, c); }

__device__ __forceinline__ int band_of(const BandArgs& B, int64_t k, int64_t N) {
  int64_t kk = k < N - 1 - k ? k : N - 1 - k;
  for (int s = 0; s < B.K; ++s)
    if (kk >= B.ka[s] && kk < B.kb[s]) return s;
  return -1;
}

// FP32 band vectors of FP64 plans are scaled by exact powers of two: 2^{e_sm - E}
// with e_sm a per-(band, term) exponent of the plan (so that the largest entry
// of the vector is about 1 for unit input) and E the exponent of the item's
// largest input magnitude; the epilogues undo it in FP64.
struct Scale32 {
  const int* e;                         // [2][K][M]: forward, transposed
  const unsigned long long* amax;       // [item] bits of max |input| (a non-negative double)
  const float* H32;                     // [M - Mh][N]: C_n h_{m,n} 2^{e_{K-1,m}} (0 below the last cut)
  const ffd* Hff;                       // [Mh - M64][N]: the same for the float-float terms
};
__device__ __forceinline__ double pow2i(int e) {
  e = max(-1022, min(1023, e));
  return __longlong_as_double((long long)(1023 + e) << 52);
}
// Conversions between double and float built from the bit patterns.  On GB300 a
// double <-> float conversion instruction issues on the FP64 pipe (measured 595
// G/s, the DFMA rate, against 11 T/s for int -> float), and the stage kernels of
// FP64 plans convert at every boundary between their FP64 and FP32-pipe tiers, so
// they assemble the IEEE 754 fields with integer operations instead.  Values are
// scaled to magnitudes near 1 by exact powers of two before they are converted;
// floats below the normal range (2^-126) are flushed to zero.

// v 2^e by exponent-field arithmetic (exact); zero stays zero, results below the
// double normal range flush to zero (|v 2^e| < 2^1024 is the caller's)
__device__ __forceinline__ double scale2(double v, int e) {
  const long long b = __double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0 || E + e <= 0) return __longlong_as_double(b & (long long)0x8000000000000000ull);
  return __longlong_as_double(b + ((long long)e << 52));
}
// float nearest to v (ties away from zero); |v| >= 2^128 gives infinity
__device__ __forceinline__ float f32_of(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long a = b & 0x7fffffffffffffffull;
  const unsigned int sg = (unsigned int)(b >> 32) & 0x80000000u;
  if (a < (897ull << 52)) return __uint_as_float(sg);
  if (a >= (1151ull << 52)) return __uint_as_float(sg | 0x7f800000u);
  return __uint_as_float(sg | (unsigned int)(((a + (1ull << 28)) >> 29) - (896ull << 23)));
}
// double of a float (exact; subnormal floats give zero)
__device__ __forceinline__ double f64_of(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned long long a = u & 0x7fffffffu;
  const unsigned long long sg = (unsigned long long)(u & 0x80000000u) << 32;
  if (a < 0x00800000ull) return __longlong_as_double((long long)sg);
  return __longlong_as_double((long long)(sg | ((a + (896ull << 23)) << 29)));
}
// float-float pair of a double: hi = v rounded to float, lo = v - hi (an integer
// of at most 29 bits in units of 2^(E-1075), E the biased exponent of v) rounded
// to float; the pair carries v to 2^-48 relative
__device__ __forceinline__ ffd ffd_of(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long a = b & 0x7fffffffffffffffull;
  const unsigned int sg = (unsigned int)(b >> 32) & 0x80000000u;
  if (a < (897ull << 52)) return ffd(0.f, 0.f);
  if (a >= (1151ull << 52)) return ffd(__uint_as_float(sg | 0x7f800000u), 0.f);
  const unsigned long long up = (a >> 28) & 1ull;
  const unsigned int hb = (unsigned int)((a >> 29) + up - (896ull << 23));
  const int rem = (int)(a & ((1ull << 29) - 1ull)) - (int)(up << 29);  // |rem| <= 2^28
  const int E = (int)(a >> 52);  // 897 <= E <= 1150 here
  // rem 2^(E-1075); below E = 949 that power is not a normal float, so it is
  // applied as 2^(E-1011) 2^-64
  const bool big = E >= 949;
  const float sc = __uint_as_float((unsigned int)(big ? E - 948 : E - 884) << 23);
  const float lo = __int2float_rn(rem) * sc * (big ? 1.f : 0x1p-64f);
  return ffd(__uint_as_float(sg | hb), sg ? -lo : lo);
}
__device__ __forceinline__ ffc ffc_of(double x, double y) {
  ffc r;
  r.x = ffd_of(x);
  r.y = ffd_of(y);
  return r;
}
// hi + lo in double: one FP64 addition
__device__ __forceinline__ double dbl_of(ffd a) { return f64_of(a.hi) + f64_of(a.lo); }
// an index 0 <= n <= 2^24 (every N of a plan) in precision T; exact, and for
// double without the FP64-pipe conversion instruction
template <typename T>
__device__ __forceinline__ T idx_t(int64_t n) {
  if constexpr (is_f64<T>) {
    return f64_of(__int2float_rn((int)n));
  } else {
    return (T)n;
  }
}

// 2^e as a float (e clamped to the normal range)
__device__ __forceinline__ float pow2f(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((127 + e) << 23);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ int item_exp(const Scale32& S, int64_t bt) {
  const unsigned long long b = S.amax[bt];
  return b == 0ull ? 0 : (int)((b >> 52) & 0x7ff) - 1023;
}

// 1/l for the Taylor coefficients t^l / l! (products instead of divisions)
__constant__ double kInvInt[48] = {
    0.0,        1.0,        1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,  1.0 / 9,
    1.0 / 10,   1.0 / 11,   1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19,
    1.0 / 20,   1.0 / 21,   1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29,
    1.0 / 30,   1.0 / 31,   1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39,
    1.0 / 40,   1.0 / 41,   1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47};

// 1/((l+1)(l+2)): q_{l+2} = q_l t^2 / ((l+1)(l+2)) in one product per term
#define GB_INVP(l) 1.0 / (((l) + 1.0) * ((l) + 2.0))
__constant__ double kInvPair[46] = {
    GB_INVP(0),  GB_INVP(1),  GB_INVP(2),  GB_INVP(3),  GB_INVP(4),  GB_INVP(5),  GB_INVP(6),  GB_INVP(7),
    GB_INVP(8),  GB_INVP(9),  GB_INVP(10), GB_INVP(11), GB_INVP(12), GB_INVP(13), GB_INVP(14), GB_INVP(15),
    GB_INVP(16), GB_INVP(17), GB_INVP(18), GB_INVP(19), GB_INVP(20), GB_INVP(21), GB_INVP(22), GB_INVP(23),
    GB_INVP(24), GB_INVP(25), GB_INVP(26), GB_INVP(27), GB_INVP(28), GB_INVP(29), GB_INVP(30), GB_INVP(31),
    GB_INVP(32), GB_INVP(33), GB_INVP(34), GB_INVP(35), GB_INVP(36), GB_INVP(37), GB_INVP(38), GB_INVP(39),
    GB_INVP(40), GB_INVP(41), GB_INVP(42), GB_INVP(43), GB_INVP(44), GB_INVP(45)};
#undef GB_INVP

// the same 1/l as float-float pairs (the float-float Taylor pairs)
#define GB_FFINV(l) ffd(1.0 / (l))
__constant__ ffd kInvIntFF[48] = {
    ffd(0.f, 0.f), GB_FFINV(1),  GB_FFINV(2),  GB_FFINV(3),  GB_FFINV(4),  GB_FFINV(5),  GB_FFINV(6),
    GB_FFINV(7),   GB_FFINV(8),  GB_FFINV(9),  GB_FFINV(10), GB_FFINV(11), GB_FFINV(12), GB_FFINV(13),
    GB_FFINV(14),  GB_FFINV(15), GB_FFINV(16), GB_FFINV(17), GB_FFINV(18), GB_FFINV(19), GB_FFINV(20),
    GB_FFINV(21),  GB_FFINV(22), GB_FFINV(23), GB_FFINV(24), GB_FFINV(25), GB_FFINV(26), GB_FFINV(27),
    GB_FFINV(28),  GB_FFINV(29), GB_FFINV(30), GB_FFINV(31), GB_FFINV(32), GB_FFINV(33), GB_FFINV(34),
    GB_FFINV(35),  GB_FFINV(36), GB_FFINV(37), GB_FFINV(38), GB_FFINV(39), GB_FFINV(40), GB_FFINV(41),
    GB_FFINV(42),  GB_FFINV(43), GB_FFINV(44), GB_FFINV(45), GB_FFINV(46), GB_FFINV(47)};
#undef GB_FFINV
// x times an exact power-of-two float (no rounding)
__device__ __forceinline__ ffd ff_scale(ffd x, float p) { return ffd(x.hi * p, x.lo * p); }

// signed Taylor coefficient of the cos part ((-1)^{l/2}, l even) and of the sin
// part ((-1)^{(l+1)/2}, l odd), Eq. (6)
__device__ __forceinline__ int sgn_even(int l) { return ((l >> 1) & 1) ? -1 : 1; }
__device__ __forceinline__ int sgn_odd(int l) { return (((l + 1) >> 1) & 1) ? -1 : 1; }

// ---------------------------------------------------------------- leg2cheb
// C_n h_{m,n} for term m: from the plan's table in FP64 (Hnm[m N + n]); the FP32
// form runs the recurrence h_{m+1} = h_m (m+1/2)^2 / ((m+1)(n+m+3/2)) in float
template <typename T>
struct HTerm {
  const double* Hnm;
  int64_t N, n;
  T cn, h;
  __device__ __forceinline__ T at(int m) {
    if constexpr (sizeof(T) == 8) {
      return Hnm[(int64_t)m * N + n];
    } else {
      const T v = cn * h;
      const T mh = (T)m + (T)0.5;
      h = h * (mh * mh) / (((T)m + (T)1) * ((T)n + (T)m + (T)1.5));
      return v;
    }
  }
};

// terms m < Mh go to U ([band][m][N], precision T), terms m >= Mh to U32
// ([band][m - Mh][N], FP32)
template <typename T>
__global__ void k_l2c_pro(const T* __restrict__ c, C2<T>* __restrict__ U, ffc* __restrict__ Uff,
                          float2* __restrict__ U32, int64_t N, int M, int Mh, int M64, BandArgs B,
                          const double* __restrict__ Cn, const double* __restrict__ Hnm, TwArgs<T> tw4N,
                          Scale32 S) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t bt = blockIdx.y;
  const int Ml = M - Mh, Mf = Mh - M64;
  const int E = (U32 || Uff) ? item_exp(S, bt) : 0;
  c += bt * N;
  U += bt * (int64_t)B.K * M64 * N;
  if (Uff) Uff += bt * (int64_t)B.K * Mf * N;
  if (U32) U32 += bt * (int64_t)B.K * Ml * N;
  const T cv = c[n];
  const C2<T> e = twid<T>(tw4N, n);
  const C2<T> ce = mk<T>(cv * e.x, cv * e.y);
  HTerm<T> H{Hnm, N, n, sizeof(T) == 8 ? (T)0 : (T)Cn[n], (T)1};
  const C2<T> zero = mk<T>((T)0, (T)0);
  for (int m = 0; m < M64; ++m) {
    const T a = H.at(m);
    const C2<T> val = mk<T>(a * ce.x, a * ce.y);
    for (int s = 0; s < B.K; ++s) U[(int64_t)(s * M64 + m) * N + n] = (n >= B.ns[s]) ? val : zero;
  }
  if (Mf > 0) {
    // float-float terms: Hff = C_n h_{m,n} 2^{e_{K-1,m}} times c_n e_n 2^{-E} in
    // float-float, then the band's exact 2^{e_{s,m} - e_{K-1,m}}
    const ffc cf = ffc_of(scale2((double)ce.x, -E), scale2((double)ce.y, -E));
    const int* eK = S.e + (B.K - 1) * M;
    const ffc zz = {ffd(0.f, 0.f), ffd(0.f, 0.f)};
    for (int m = M64; m < Mh; ++m) {
      const ffd h = S.Hff[(int64_t)(m - M64) * N + n];
      const ffd vx = h * cf.x, vy = h * cf.y;
      for (int s = 0; s < B.K; ++s) {
        const float p = pow2f(S.e[s * M + m] - eK[m]);
        ffc w;
        w.x = ffd(vx.hi * p, vx.lo * p);
        w.y = ffd(vy.hi * p, vy.lo * p);
        Uff[(int64_t)(s * Mf + m - M64) * N + n] = (n >= B.ns[s]) ? w : zz;
      }
    }
  }
  if (Ml > 0) {
    // FP32 terms: C_n h_{m,n} 2^{e_{s,m}} c_n e_n 2^{-E} from the float table
    // H32 = C_n h_{m,n} 2^{e_{K-1,m}} times the band's exact 2^{e_{s,m} - e_{K-1,m}}
    const float2 cf = make_float2(f32_of(scale2((double)ce.x, -E)), f32_of(scale2((double)ce.y, -E)));
    const int* eK = S.e + (B.K - 1) * M;
    for (int m = Mh; m < M; ++m) {
      const float h32 = S.H32[(int64_t)(m - Mh) * N + n];
      for (int s = 0; s < B.K; ++s) {
        const float a = h32 * pow2f(S.e[s * M + m] - eK[m]);
        U32[(int64_t)(s * Ml + m - Mh) * N + n] =
            (n >= B.ns[s]) ? make_float2(a * cf.x, a * cf.y) : make_float2(0.f, 0.f);
      }
    }
  }
}

// Per cheb1 row k: alpha_k = e^{i(theta_k/2 - pi/4)} / (2 sin theta_k)^{1/2} and
// rho_k = e^{i(theta_k - pi/2)} / (2 sin theta_k), so that the term-m factor
// e^{i(m+1/2)(theta_k - pi/2)} / (2 sin theta_k)^{m+1/2} is alpha_k rho_k^m.  FP64
// plans read them from a table (AR[k] = {alpha, rho}); the FP32 form computes them.
template <typename T>
__device__ __forceinline__ void row_factors(int64_t k, int64_t N, const RowAR* __restrict__ AR, C2<T>& al,
                                            C2<T>& rho) {
  if constexpr (sizeof(T) == 8) {
    const RowAR a = AR[k];
    al = mk<T>(a.ax, a.ay);
    rho = mk<T>(a.rx, a.ry);
  } else {
    T st, ct, sa, ca;
    sincospi_t((T)(2 * k + 1) / (T)(2 * N), &st, &ct);      // theta_k
    sincospi_t((T)(2 * k + 1 - N) / (T)(4 * N), &sa, &ca);  // theta_k/2 - pi/4
    const T g = (T)0.5 / st;
    const T sq = sqrt(g);
    al = mk<T>(ca * sq, sa * sq);
    rho = mk<T>(st * g, -ct * g);
  }
}

__global__ void k_row_factors_init(RowAR* __restrict__ AR, int64_t N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double st, ct, sa, ca;
  sincospi((double)(2 * k + 1) / (double)(2 * N), &st, &ct);
  sincospi((double)(2 * k + 1 - N) / (double)(4 * N), &sa, &ca);
  const double g = 0.5 / st;
  const double sq = sqrt(g);
  AR[k] = RowAR{ca * sq, sa * sq, st * g, -ct * g};
}

// Hnm[m N + n] = C_n h_{m,n} for the FP64 terms m < M64 (the recurrence in FP64,
// once per plan); for the float-float terms M64 <= m < Mh and the FP32 terms
// m >= Mh, Hff[(m - M64) N + n] and H32[(m - Mh) N + n] = C_n h_{m,n} 2^{eK[m]},
// 0 below the smallest band cut ns_min (never read there)
__global__ void k_hnm_init(double* __restrict__ Hnm, ffd* __restrict__ Hff, float* __restrict__ H32,
                           const double* __restrict__ Cn, int64_t N, int M, int Mh, int M64,
                           const int* __restrict__ eK, int64_t ns_min) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double h = 1.0;
  const double cn = Cn[n];
  for (int m = 0; m < M; ++m) {
    if (m < M64)
      Hnm[(int64_t)m * N + n] = cn * h;
    else if (m < Mh)
      Hff[(int64_t)(m - M64) * N + n] = n >= ns_min ? ffd_of(cn * h * pow2i(eK[m])) : ffd(0.f, 0.f);
    else
      H32[(int64_t)(m - Mh) * N + n] = n >= ns_min ? (float)(cn * h * pow2i(eK[m])) : 0.f;
    const double mh = (double)m + 0.5;
    h = h * (mh * mh) / (((double)m + 1.0) * ((double)n + (double)m + 1.5));
  }
}

template <typename T>
__global__ void k_l2c_epi(const C2<T>* __restrict__ Y, const ffc* __restrict__ Yff, const float2* __restrict__ Y32,
                          const T* __restrict__ vrec, T* __restrict__ v, int64_t N, int M, int Mh, int M64,
                          BandArgs B, const RowAR* __restrict__ AR, Scale32 S) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int64_t bt = blockIdx.y;
  const int Ml = M - Mh, Mf = Mh - M64;
  vrec += bt * N;
  v += bt * N;
  if (Y) Y += bt * (int64_t)B.K * M64 * N;
  if (Yff) Yff += bt * (int64_t)B.K * Mf * N;
  if (Y32) Y32 += bt * (int64_t)B.K * Ml * N;
  T acc = vrec[k];
  const int s = band_of(B, k, N);
  if (s >= 0) {
    C2<T> al, rho;
    row_factors<T>(k, N, AR, al, rho);
    const bool odd = k & 1;
    const int64_t idx = odd ? N - 1 - (k >> 1) : (k >> 1);
    const C2<T>* y = Y + (int64_t)s * M64 * N + idx;
    for (int m = 0; m < M64; ++m) {
      C2<T> z = y[(int64_t)m * N];
      if (odd) z.y = -z.y;
      acc += al.x * z.x - al.y * z.y;
      al = cmul<T>(al, rho);
    }
    // al = alpha rho^M64 here
    ffc bff;  // float-float b_m = alpha rho^m 2^{-e_{s,m}}
    if (Mf > 0) {
      // float-float terms: with the band's FFT output scaled by 2^{e_{s,m} - E},
      // term m adds 2^E Re(b_m z_m); b advances by rho 2^{e_{s,m} - e_{s,m+1}}
      const int* e = S.e + s * M;
      bff = ffc_of(scale2((double)al.x, -e[M64]), scale2((double)al.y, -e[M64]));
      const ffc r = ffc_of((double)rho.x, (double)rho.y);
      ffd aff(0.f, 0.f);
      for (int m = M64; m < Mh; ++m) {
        ffc z = Yff[(int64_t)(s * Mf + m - M64) * N + idx];
        if (odd) z.y = -z.y;
        aff = aff + ff_dot2(bff.x, z.x, bff.y, z.y, -1.f);
        if (m + 1 < M) {
          const float p = pow2f(e[m] - e[m + 1]);
          ffc rp;
          rp.x = ffd(r.x.hi * p, r.x.lo * p);
          rp.y = ffd(r.y.hi * p, r.y.lo * p);
          bff = cmul<ffd>(bff, rp);
        }
      }
      acc += (T)scale2(dbl_of(aff), item_exp(S, bt));
    }
    if (Ml > 0) {
      // FP32 terms: with the band's FFT output scaled by 2^{e_{s,m} - E}, term m
      // adds 2^E Re(b_m z_m), b_m = alpha rho^m 2^{-e_{s,m}}, continued from the
      // float-float terms (or from al = alpha rho^Mh when there are none)
      const int* e = S.e + s * M;
      float2 b;
      if (Mf > 0) {
        b = make_float2(bff.x.hi, bff.y.hi);
      } else {
        b = make_float2(f32_of(scale2((double)al.x, -e[Mh])), f32_of(scale2((double)al.y, -e[Mh])));
      }
      const float2 r = make_float2(f32_of((double)rho.x), f32_of((double)rho.y));
      const float2* y32 = Y32 + (int64_t)s * Ml * N + idx;
      float a32 = 0.f;
      for (int m = Mh; m < M; ++m) {
        float2 z = y32[(int64_t)(m - Mh) * N];
        if (odd) z.y = -z.y;
        a32 = fmaf(b.x, z.x, fmaf(-b.y, z.y, a32));
        if (m + 1 < M) {
          const float p = pow2f(e[m] - e[m + 1]);
          b = cmulf(b, make_float2(r.x * p, r.y * p));
        }
      }
      acc += (T)scale2(f64_of(a32), item_exp(S, bt));
    }
  }
  v[k] = acc;
}

// ---------------------------------------------------------------- A4: values -> coefficients
template <typename T>
__global__ void k_a4_pro(const T* __restrict__ v, C2<T>* __restrict__ U, int64_t N) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= N / 2) return;
  v += (int64_t)blockIdx.y * N;
  U += (int64_t)blockIdx.y * N;
  U[kp] = mk<T>(v[2 * kp], (T)0);
  U[N - 1 - kp] = mk<T>(v[2 * kp + 1], (T)0);
}

template <typename T>
__global__ void k_a4_epi(const C2<T>* __restrict__ F, T* __restrict__ chat, int64_t N, T invN, TwArgs<T> tw4N,
                         const double* __restrict__ hb, int64_t h, int64_t hs) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  F += (int64_t)blockIdx.y * N;
  chat += (int64_t)blockIdx.y * N;
  const C2<T> Fn = F[n];
  const C2<T> Fm = F[(N - n) & (N - 1)];
  const C2<T> Vh = mk<T>((Fn.x + Fm.x) * (T)0.5, (Fn.y - Fm.y) * (T)0.5);
  const C2<T> e = twid<T>(tw4N, n);  // conj(e) = e^{-i pi n/(2N)}
  const T U = e.x * Vh.x + e.y * Vh.y;
  const T a = (n == 0 ? invN : (T)2 * invN) * U;
  // the head block's columns (when it ran beside this chain): added in double
  chat[n] = (hb && n < h) ? (T)((double)a + hb[(int64_t)blockIdx.y * hs + n]) : a;
}

// ---------------------------------------------------------------- FCS helpers
template <typename T>
__global__ void k_fcs_pro(const T* __restrict__ a, C2<T>* __restrict__ U, int64_t N, int scale_d, T invN,
                          TwArgs<T> tw4N) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  a += (int64_t)blockIdx.y * N;
  U += (int64_t)blockIdx.y * N;
  T an = a[n];
  if (scale_d) an *= n == 0 ? invN : (T)2 * invN;
  const C2<T> e = twid<T>(tw4N, n);
  U[n] = mk<T>(an * e.x, an * e.y);
}

template <typename T>
__global__ void k_fcs_re_epi(const C2<T>* __restrict__ Y, T* __restrict__ out, int64_t N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  Y += (int64_t)blockIdx.y * N;
  out += (int64_t)blockIdx.y * N;
  const int64_t idx = (k & 1) ? N - 1 - (k >> 1) : (k >> 1);
  out[k] = Y[idx].x;
}

// ---------------------------------------------------------------- Taylor (forward)
// pair p: X part l_a = 2p + (inc0 ? 0 : 2), Y part l_b = 2p + 1; a term is used
// only when its l <= L-1.
// pairs p < P64 go to U ([item][P64][N], precision T), pairs p >= P64 to Uff
// ([item][npair - P64][N], float-float, scaled by 2^{-E})
template <typename T>
__global__ void k_tay_pro(const T* __restrict__ chat, C2<T>* __restrict__ U, ffc* __restrict__ Uff, int64_t N,
                          int L, int inc0, int npair, int P64, T invN, TwArgs<T> tw4N, Scale32 S) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t bt = blockIdx.y;
  chat += bt * N;
  U += bt * P64 * N;
  if (Uff) Uff += bt * (npair - P64) * N;
  const T r = idx_t<T>(n) * invN;  // exact: N is a power of two
  const T rN = idx_t<T>(N - n) * invN;
  const T cn = chat[n];
  const T cm = n > 0 ? chat[N - n] : (T)0;
  const C2<T> e = twid<T>(tw4N, n);
  // U_n = e_n [(a_n + b_n) - i (a_{N-n} - b_{N-n})] with a = r^{l_a} chat, b = r^{l_b} chat:
  // = (r^{l_a} + r^{l_b}) e chat_n + (rN^{l_b} - rN^{l_a}) i e chat_{N-n}
  const C2<T> E1 = mk<T>(e.x * cn, e.y * cn);
  const C2<T> E2 = mk<T>(-e.y * cm, e.x * cm);
  // r^l and rN^l for the current pair, advanced by r^2 per pair
  const T r2 = r * r, rN2 = rN * rN;
  T pa = inc0 ? (T)1 : r2, paN = inc0 ? (T)1 : rN2;  // r^{l_a}
  T pb = r, pbN = rN;                               // r^{l_b}
  for (int p = 0; p < P64; ++p) {
    const int la = 2 * p + (inc0 ? 0 : 2);
    const int lb = 2 * p + 1;
    const bool ua = la <= L - 1, ub = lb <= L - 1;
    C2<T> val;
    if (n == 0) {
      val = mk<T>(ua ? (T)2 * pa * cn : (T)0, (T)0);  // 0^0 = 1 for l_a = 0
    } else {
      const T A = (ua ? pa : (T)0) + (ub ? pb : (T)0);
      const T Bm = (ub ? pbN : (T)0) - (ua ? paN : (T)0);
      val = mk<T>(A * E1.x + Bm * E2.x, A * E1.y + Bm * E2.y);
    }
    U[(int64_t)p * N + n] = val;
    pa *= r2;
    paN *= rN2;
    pb *= r2;
    pbN *= rN2;
  }
  if (P64 < npair) {
    // float-float pairs: the same sums, continued from the powers reached above
    // (r = n/N and rN are exact floats, so r^2 and rN^2 are exact float-float)
    const int E = item_exp(S, bt);
    const ffc e1 = ffc_of(scale2((double)E1.x, -E), scale2((double)E1.y, -E));
    const ffc e2 = ffc_of(scale2((double)E2.x, -E), scale2((double)E2.y, -E));
    const ffd c0 = ffd_of(scale2((double)cn, -E));
    const ffd fr(f32_of((double)r), 0.f), frN(f32_of((double)rN), 0.f);
    const ffd fr2 = fr * fr, frN2 = frN * frN;
    ffd fa = ffd_of((double)pa), faN = ffd_of((double)paN), fb = ffd_of((double)pb), fbN = ffd_of((double)pbN);
    const ffd z(0.f, 0.f);
    for (int p = P64; p < npair; ++p) {
      const int la = 2 * p + (inc0 ? 0 : 2);
      const int lb = 2 * p + 1;
      const bool ua = la <= L - 1, ub = lb <= L - 1;
      ffc val;
      if (n == 0) {
        val.x = ua ? ff_scale(fa * c0, 2.f) : z;
        val.y = z;
      } else {
        const ffd A = (ua ? fa : z) + (ub ? fb : z);
        const ffd Bm = (ub ? fbN : z) - (ua ? faN : z);
        val.x = ff_dot2(A, e1.x, Bm, e2.x, 1.f);
        val.y = ff_dot2(A, e1.y, Bm, e2.y, 1.f);
      }
      Uff[(int64_t)(p - P64) * N + n] = val;
      fa = fa * fr2;
      faN = faN * frN2;
      fb = fb * fr2;
      fbN = fbN * frN2;
    }
  }
}

// GRID: the rows are those of a rule of R.n <= N nodes placed on this grid of N
// points (grid.cu; one rule per batch item): row k reads the sums at its grid
// point j = R.j[k], and R.t[k] is its offset N (theta_k - theta'_j) from that
// point; f keeps the grid's batch stride N.
template <typename T, bool GRID = false>
__global__ void k_tay_epi(const C2<T>* __restrict__ Y, const ffc* __restrict__ Yff, const T* __restrict__ v,
                          T* __restrict__ f, const double* __restrict__ tN, int64_t N, int L, int inc0, int npair,
                          int P64, Scale32 S, const GridRule* __restrict__ rules = nullptr,
                          const int32_t* __restrict__ item = nullptr) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t bt = blockIdx.y;
  GridRule R{};
  if constexpr (GRID) R = rules[item ? item[bt] : 0];
  if (k >= (GRID ? R.n : N)) return;
  Y += bt * P64 * N;
  if (Yff) Yff += bt * (npair - P64) * N;
  f += bt * N;
  if (v) v += bt * N;
  const T t = (T)(GRID ? R.t[k] : tN[k]);
  const int64_t j = GRID ? (int64_t)R.j[k] : k;
  const bool odd = j & 1;
  const int64_t idx = odd ? N - 1 - (j >> 1) : (j >> 1);
  T acc2 = (T)0;  // twice the sum of the pairs in the plan's precision
  // q_l = t^l / l! advanced term by term: pair p uses l_b = 2p+1 and l_a = 2p (inc0)
  // or 2p+2, so l runs upwards through both parts
  T qa = (T)1;                        // q_{l_a} (inc0: q_0)
  T qb = t;                           // q_{l_b} = q_1
  const T t2 = t * t;
  if (!inc0) qa = qb * t * (T)kInvInt[2];
  for (int p = 0; p < P64; ++p) {
    const int la = 2 * p + (inc0 ? 0 : 2);
    const int lb = 2 * p + 1;
    const C2<T> y = Y[(int64_t)p * N + idx];
    if (la <= L - 1) acc2 = fma(sgn_even(la) > 0 ? qa : -qa, y.x, acc2);
    if (lb <= L - 1) acc2 = fma((sgn_odd(lb) > 0) != odd ? qb : -qb, y.y, acc2);
    // next pair: l_b + 2 and l_a + 2
    if (inc0) {
      qb = qb * (t2 * (T)kInvPair[lb]);
      qa = qa * (t2 * (T)kInvPair[la]);
    } else {
      qb = qa * t * (T)kInvInt[la + 1];
      qa = qb * t * (T)kInvInt[la + 2];
    }
  }
  T acc = inc0 ? (T)0 : v[j];
  acc = fma((T)0.5, acc2, acc);
  if (P64 < npair) {
    // float-float pairs, continued from q reached above; outputs scaled by 2^{-E}
    const ffd ft = ffd_of((double)t);
    ffd fqa = ffd_of((double)qa), fqb = ffd_of((double)qb), aff(0.f, 0.f);
    const float fsk = odd ? -0.5f : 0.5f;
    for (int p = P64; p < npair; ++p) {
      const int la = 2 * p + (inc0 ? 0 : 2);
      const int lb = 2 * p + 1;
      const ffc y = Yff[(int64_t)(p - P64) * N + idx];
      if (la <= L - 1) aff = aff + ff_scale(fqa * y.x, sgn_even(la) * 0.5f);
      if (lb <= L - 1) aff = aff + ff_scale(fqb * y.y, sgn_odd(lb) * fsk);
      if (inc0) {
        fqb = fqb * ft * kInvIntFF[lb + 1] * ft * kInvIntFF[lb + 2];
        fqa = fqa * ft * kInvIntFF[la + 1] * ft * kInvIntFF[la + 2];
      } else {
        fqb = fqa * ft * kInvIntFF[la + 1];
        fqa = fqb * ft * kInvIntFF[la + 2];
      }
    }
    acc += (T)scale2(dbl_of(aff), item_exp(S, bt));
  }
  f[k] = acc;
}

// ---------------------------------------------------------------- Taylor (transposed)
template <typename T>
__global__ void k_tayt_pro(const T* __restrict__ fin, const double* __restrict__ wscale,
                           const double* __restrict__ tN, C2<T>* __restrict__ U, ffc* __restrict__ Uff, int64_t N,
                           int L, int inc0, int npair, int P64, Scale32 S) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= N / 2) return;
  const int64_t bt = blockIdx.y;
  fin += bt * N;
  U += bt * P64 * N;
  if (Uff) Uff += bt * (npair - P64) * N;
  const int64_t k0 = 2 * kp, k1 = 2 * kp + 1;
  T g0 = fin[k0], g1 = fin[k1];
  if (wscale) {
    g0 *= (T)wscale[k0];
    g1 *= (T)wscale[k1];
  }
  const T t0 = (T)tN[k0], t1 = (T)tN[k1];
  const T t02 = t0 * t0, t12 = t1 * t1;
  T pa0 = inc0 ? (T)1 : t02, pa1 = inc0 ? (T)1 : t12;
  T pb0 = t0, pb1 = t1;
  for (int p = 0; p < P64; ++p) {
    const int la = 2 * p + (inc0 ? 0 : 2);
    const int lb = 2 * p + 1;
    const T ua = la <= L - 1 ? (T)1 : (T)0;
    const T ub = lb <= L - 1 ? (T)1 : (T)0;
    // h_k = (-1)^k b_k: k0 even, k1 odd
    U[(int64_t)p * N + kp] = mk<T>(ua * pa0 * g0, ub * pb0 * g0);
    U[(int64_t)p * N + N - 1 - kp] = mk<T>(ua * pa1 * g1, -ub * pb1 * g1);
    pa0 *= t02;
    pa1 *= t12;
    pb0 *= t02;
    pb1 *= t12;
  }
  if (P64 < npair) {
    // float-float pairs, continued from the powers reached above, scaled by 2^{-E}
    const int E = item_exp(S, bt);
    const ffd fg0 = ffd_of(scale2((double)g0, -E)), fg1 = ffd_of(scale2((double)g1, -E));
    const ffd ft0 = ffd_of((double)t0), ft1 = ffd_of((double)t1);
    const ffd ft02 = ft0 * ft0, ft12 = ft1 * ft1;
    ffd fa0 = ffd_of((double)pa0), fa1 = ffd_of((double)pa1), fb0 = ffd_of((double)pb0), fb1 = ffd_of((double)pb1);
    const ffd z(0.f, 0.f);
    for (int p = P64; p < npair; ++p) {
      const int la = 2 * p + (inc0 ? 0 : 2);
      const int lb = 2 * p + 1;
      const bool ua = la <= L - 1, ub = lb <= L - 1;
      ffc w0, w1;
      w0.x = ua ? fa0 * fg0 : z;
      w0.y = ub ? fb0 * fg0 : z;
      w1.x = ua ? fa1 * fg1 : z;
      w1.y = ub ? -(fb1 * fg1) : z;
      Uff[(int64_t)(p - P64) * N + kp] = w0;
      Uff[(int64_t)(p - P64) * N + N - 1 - kp] = w1;
      fa0 = fa0 * ft02;
      fa1 = fa1 * ft12;
      fb0 = fb0 * ft02;
      fb1 = fb1 * ft12;
    }
  }
}

// k_tayt_pro for the rows of a rule placed on this plan's grid of N points (one
// rule per batch item): grid point j collects the rows k with j(k) = j
// (kf[j] <= k < kf[j+1]; at most two, checked when the maps are built), each
// with its own offset t_k; the thread of pair jp writes grid points 2jp (to
// U[jp]) and 2jp + 1 (to U[N-1-jp], with the sign (-1)^j of its sine part) as
// k_tayt_pro does.  use_w: rows weighted by the rule's w_k.
template <typename T>
__global__ void k_tayt_pro_grid(const T* __restrict__ fin, int use_w, const GridRule* __restrict__ rules,
                                const int32_t* __restrict__ item, C2<T>* __restrict__ U, ffc* __restrict__ Uff,
                                int64_t N, int L, int inc0, int npair, int P64, Scale32 S) {
  const int64_t jp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (jp >= N / 2) return;
  const int64_t bt = blockIdx.y;
  const GridRule R = rules[item ? item[bt] : 0];
  const int32_t* __restrict__ kf = R.kf;
  const double* __restrict__ tr = R.t;
  const double* __restrict__ wscale = use_w ? R.w : nullptr;
  fin += bt * N;
  U += bt * P64 * N;
  if (Uff) Uff += bt * (npair - P64) * N;
  // slots 0, 1: the rows of grid point 2jp; slots 2, 3: those of 2jp + 1
  const int64_t ka = kf[2 * jp], kb = kf[2 * jp + 1], kc = kf[2 * jp + 2];
  T g[4], t[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t k = (s < 2 ? ka : kb) + (s & 1);
    const bool in = k < (s < 2 ? kb : kc);
    g[s] = in ? fin[k] : (T)0;
    if (in && wscale) g[s] *= (T)wscale[k];
    t[s] = in ? (T)tr[k] : (T)0;
  }
  T pa[4], pb[4], t2[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    t2[s] = t[s] * t[s];
    pa[s] = inc0 ? (T)1 : t2[s];
    pb[s] = t[s];
  }
  for (int p = 0; p < P64; ++p) {
    const int la = 2 * p + (inc0 ? 0 : 2);
    const int lb = 2 * p + 1;
    const T ua = la <= L - 1 ? (T)1 : (T)0;
    const T ub = lb <= L - 1 ? (T)1 : (T)0;
    U[(int64_t)p * N + jp] = mk<T>(ua * (pa[0] * g[0] + pa[1] * g[1]), ub * (pb[0] * g[0] + pb[1] * g[1]));
    U[(int64_t)p * N + N - 1 - jp] = mk<T>(ua * (pa[2] * g[2] + pa[3] * g[3]), -ub * (pb[2] * g[2] + pb[3] * g[3]));
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      pa[s] *= t2[s];
      pb[s] *= t2[s];
    }
  }
  if (P64 < npair) {
    // float-float pairs, continued from the powers reached above, scaled by 2^{-E}
    const int E = item_exp(S, bt);
    ffd fg[4], ft2[4], fa[4], fb[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      fg[s] = ffd_of(scale2((double)g[s], -E));
      const ffd ft = ffd_of((double)t[s]);
      ft2[s] = ft * ft;
      fa[s] = ffd_of((double)pa[s]);
      fb[s] = ffd_of((double)pb[s]);
    }
    const ffd z(0.f, 0.f);
    for (int p = P64; p < npair; ++p) {
      const int la = 2 * p + (inc0 ? 0 : 2);
      const int lb = 2 * p + 1;
      const bool ua = la <= L - 1, ub = lb <= L - 1;
      ffc w0, w1;
      w0.x = ua ? fa[0] * fg[0] + fa[1] * fg[1] : z;
      w0.y = ub ? fb[0] * fg[0] + fb[1] * fg[1] : z;
      w1.x = ua ? fa[2] * fg[2] + fa[3] * fg[3] : z;
      w1.y = ub ? -(fb[2] * fg[2] + fb[3] * fg[3]) : z;
      Uff[(int64_t)(p - P64) * N + jp] = w0;
      Uff[(int64_t)(p - P64) * N + N - 1 - jp] = w1;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        fa[s] = fa[s] * ft2[s];
        fb[s] = fb[s] * ft2[s];
      }
    }
  }
}

// Q != null: write the FCS input of A4^T, Q_n = d_n u'_n e^{i pi n/(2N)};
// uout != null: write u_n to uout for n < nu (both when the chain also needs the
// first nu coefficients of u, for the dense head block).
template <typename T>
__global__ void k_tayt_epi(const C2<T>* __restrict__ F, const ffc* __restrict__ Fff, C2<T>* __restrict__ Q,
                           T* __restrict__ uout, int64_t N, int L, int inc0, int npair, int P64, int64_t nu, T invN,
                           TwArgs<T> tw4N, Scale32 S) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t bt = blockIdx.y;
  F += bt * P64 * N;
  if (Fff) Fff += bt * (npair - P64) * N;
  if (Q) Q += bt * N;
  if (uout) uout += bt * N;
  const T r = idx_t<T>(n) * invN;  // exact: N is a power of two
  const C2<T> e = twid<T>(tw4N, n);
  const int64_t nm = (N - n) & (N - 1);
  // with U_n = Re[conj(e) (Fn + conj Fm)]/2 (DCT-II part) and
  // V_n = Re[-e (Fm - conj Fn)]/2 (DST-II part, 0 at n = 0), the sum over pairs of
  // sgn_a q_a U - sgn_b q_b V is e.x Ax + e.y Ay with
  //   Ax = sum (ca (Fn.x + Fm.x) - cb (Fm.x - Fn.x)),  Ay = sum (ca (Fn.y - Fm.y) + cb (Fm.y + Fn.y)),
  // ca = sgn_a q_a / 2, cb = sgn_b q_b / 2
  T Ax = (T)0, Ay = (T)0;
  T qa = (T)1, qb = r;  // r^l / l! for l_a (inc0: 0) and l_b = 1
  const T r2 = r * r;
  if (!inc0) qa = qb * r * (T)kInvInt[2];
  for (int p = 0; p < P64; ++p) {
    const int la = 2 * p + (inc0 ? 0 : 2);
    const int lb = 2 * p + 1;
    const C2<T> Fn = F[(int64_t)p * N + n];
    const C2<T> Fm = F[(int64_t)p * N + nm];
    // 2 ca and 2 cb (the halving is applied once, after the loop); then
    // Ax += (ca + cb) Fn.x + (ca - cb) Fm.x,  Ay += (ca + cb) Fn.y - (ca - cb) Fm.y
    const T ca2 = la <= L - 1 ? (sgn_even(la) > 0 ? qa : -qa) : (T)0;
    const T cb2 = (lb <= L - 1 && n > 0) ? (sgn_odd(lb) > 0 ? qb : -qb) : (T)0;
    const T al = ca2 + cb2, be = ca2 - cb2;
    Ax = fma(al, Fn.x, fma(be, Fm.x, Ax));
    Ay = fma(al, Fn.y, fma(-be, Fm.y, Ay));
    if (inc0) {
      qb = qb * (r2 * (T)kInvPair[lb]);
      qa = qa * (r2 * (T)kInvPair[la]);
    } else {
      qb = qa * r * (T)kInvInt[la + 1];
      qa = qb * r * (T)kInvInt[la + 2];
    }
  }
  Ax *= (T)0.5;
  Ay *= (T)0.5;
  if (P64 < npair) {
    // float-float pairs (outputs scaled by 2^{-E}), continued from q reached above
    const ffd fr(f32_of((double)r), 0.f);  // n/N: exact
    ffd fqa = ffd_of((double)qa), fqb = ffd_of((double)qb);
    ffd ax(0.f, 0.f), ay(0.f, 0.f);
    for (int p = P64; p < npair; ++p) {
      const int la = 2 * p + (inc0 ? 0 : 2);
      const int lb = 2 * p + 1;
      const ffc Fn = Fff[(int64_t)(p - P64) * N + n];
      const ffc Fm = Fff[(int64_t)(p - P64) * N + nm];
      const float ha = la <= L - 1 ? (sgn_even(la) > 0 ? 0.5f : -0.5f) : 0.f;
      const float hb = (lb <= L - 1 && n > 0) ? (sgn_odd(lb) > 0 ? 0.5f : -0.5f) : 0.f;
      const ffd ca = ff_scale(fqa, ha), cb = ff_scale(fqb, hb);
      ax = ax + ff_dot2(ca, Fn.x + Fm.x, cb, Fm.x - Fn.x, -1.f);
      ay = ay + ff_dot2(ca, Fn.y - Fm.y, cb, Fm.y + Fn.y, 1.f);
      if (inc0) {
        fqb = fqb * fr * kInvIntFF[lb + 1] * fr * kInvIntFF[lb + 2];
        fqa = fqa * fr * kInvIntFF[la + 1] * fr * kInvIntFF[la + 2];
      } else {
        fqb = fqa * fr * kInvIntFF[la + 1];
        fqa = fqb * fr * kInvIntFF[la + 2];
      }
    }
    const int E = item_exp(S, bt);
    Ax += (T)scale2(dbl_of(ax), E);
    Ay += (T)scale2(dbl_of(ay), E);
  }
  const T acc = e.x * Ax + e.y * Ay;
  if (Q) {
    const T d = n == 0 ? invN : (T)2 * invN;
    const T a = d * acc;
    Q[n] = mk<T>(a * e.x, a * e.y);
  }
  if (uout && n < nu) uout[n] = acc;
}

// ---------------------------------------------------------------- leg2cheb (transposed)
// Per row: z_k = [g_k] + Re Z_k (A4^T output, when Y != null); then for its band
// s and each m the T2 input beta = z_k alpha_{m,k} (alpha as in the forward
// combine) is written for (s, m) and zeros for every other band.
template <typename T>
__device__ __forceinline__ T row_z(const C2<T>* Y, const T* g, const double* wscale, int64_t k,
                                   int64_t N) {
  T z = (T)0;
  if (g) {
    z = g[k];
    if (wscale) z *= (T)wscale[k];
  }
  if (Y) {
    const int64_t idx = (k & 1) ? N - 1 - (k >> 1) : (k >> 1);
    z += Y[idx].x;
  }
  return z;
}

template <typename T>
__global__ void k_l2ct_pro(const C2<T>* __restrict__ Y, const T* __restrict__ g,
                           const double* __restrict__ wscale, T* __restrict__ zout,
                           C2<T>* __restrict__ U, ffc* __restrict__ Uff, float2* __restrict__ U32, int64_t N,
                           int M, int Mh, int M64, BandArgs B, const RowAR* __restrict__ AR, Scale32 S) {
  const int64_t kp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (kp >= N / 2) return;
  const int64_t bt = blockIdx.y;
  const int Ml = M - Mh, Mf = Mh - M64;
  if (Y) Y += bt * N;
  if (g) g += bt * N;
  zout += bt * N;
  U += bt * (int64_t)B.K * M64 * N;
  if (Uff) Uff += bt * (int64_t)B.K * Mf * N;
  if (U32) U32 += bt * (int64_t)B.K * Ml * N;
  const int64_t k0 = 2 * kp, k1 = 2 * kp + 1;
  const T z0 = row_z<T>(Y, g, wscale, k0, N);
  const T z1 = row_z<T>(Y, g, wscale, k1, N);
  zout[k0] = z0;
  zout[k1] = z1;
  const int s0 = band_of(B, k0, N), s1 = band_of(B, k1, N);
  C2<T> al0 = mk<T>(0, 0), rho0 = mk<T>(0, 0), al1 = mk<T>(0, 0), rho1 = mk<T>(0, 0);
  if (s0 >= 0) row_factors<T>(k0, N, AR, al0, rho0);
  if (s1 >= 0) row_factors<T>(k1, N, AR, al1, rho1);
  for (int m = 0; m < M64; ++m) {
    // beta = z alpha; a = Re beta, h = (-1)^k Im beta
    const C2<T> v0 = mk<T>(z0 * al0.x, z0 * al0.y);
    const C2<T> v1 = mk<T>(z1 * al1.x, -z1 * al1.y);
    for (int s = 0; s < B.K; ++s) {
      C2<T>* u = U + (int64_t)(s * M64 + m) * N;
      u[kp] = (s == s0) ? v0 : mk<T>(0, 0);
      u[N - 1 - kp] = (s == s1) ? v1 : mk<T>(0, 0);
    }
    if (s0 >= 0) al0 = cmul<T>(al0, rho0);
    if (s1 >= 0) al1 = cmul<T>(al1, rho1);
  }
  // al = alpha rho^M64 here.  The float-float and FP32 terms write
  // beta 2^{g_{s,m} - E} = (z 2^{-E}) gamma_m with gamma_m = alpha rho^m 2^{g_{s,m}},
  // advanced by rho 2^{g_{s,m+1} - g_{s,m}} (float-float, then FP32)
  if (Mf > 0 || Ml > 0) {
    const int E = item_exp(S, bt);
    const int* g0 = S.e + B.K * M + max(s0, 0) * M;
    const int* g1 = S.e + B.K * M + max(s1, 0) * M;
    const ffc zz = {ffd(0.f, 0.f), ffd(0.f, 0.f)};
    ffc c0ff = zz, c1ff = zz;
    if (Mf > 0) {
      const ffd f0 = ffd_of(scale2((double)z0, -E)), f1 = ffd_of(scale2((double)z1, -E));
      ffc r0 = zz, r1 = zz;
      if (s0 >= 0) {
        c0ff = ffc_of(scale2((double)al0.x, g0[M64]), scale2((double)al0.y, g0[M64]));
        r0 = ffc_of((double)rho0.x, (double)rho0.y);
      }
      if (s1 >= 0) {
        c1ff = ffc_of(scale2((double)al1.x, g1[M64]), scale2((double)al1.y, g1[M64]));
        r1 = ffc_of((double)rho1.x, (double)rho1.y);
      }
      for (int m = M64; m < Mh; ++m) {
        ffc w0, w1;
        w0.x = f0 * c0ff.x;
        w0.y = f0 * c0ff.y;
        w1.x = f1 * c1ff.x;
        w1.y = -(f1 * c1ff.y);
        for (int s = 0; s < B.K; ++s) {
          ffc* u = Uff + (int64_t)(s * Mf + m - M64) * N;
          u[kp] = (s == s0) ? w0 : zz;
          u[N - 1 - kp] = (s == s1) ? w1 : zz;
        }
        if (m + 1 < M) {
          const float p0 = pow2f(g0[m + 1] - g0[m]), p1 = pow2f(g1[m + 1] - g1[m]);
          ffc q0, q1;
          q0.x = ffd(r0.x.hi * p0, r0.x.lo * p0);
          q0.y = ffd(r0.y.hi * p0, r0.y.lo * p0);
          q1.x = ffd(r1.x.hi * p1, r1.x.lo * p1);
          q1.y = ffd(r1.y.hi * p1, r1.y.lo * p1);
          c0ff = cmul<ffd>(c0ff, q0);
          c1ff = cmul<ffd>(c1ff, q1);
        }
      }
    }
    if (Ml > 0) {
      const float f0 = f32_of(scale2((double)z0, -E)), f1 = f32_of(scale2((double)z1, -E));
      float2 c0 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f), r0 = c0, r1 = c0;
      if (s0 >= 0) {
        if (Mf > 0) {
          c0 = make_float2(c0ff.x.hi, c0ff.y.hi);
        } else {
          c0 = make_float2(f32_of(scale2((double)al0.x, g0[Mh])), f32_of(scale2((double)al0.y, g0[Mh])));
        }
        r0 = make_float2(f32_of((double)rho0.x), f32_of((double)rho0.y));
      }
      if (s1 >= 0) {
        if (Mf > 0) {
          c1 = make_float2(c1ff.x.hi, c1ff.y.hi);
        } else {
          c1 = make_float2(f32_of(scale2((double)al1.x, g1[Mh])), f32_of(scale2((double)al1.y, g1[Mh])));
        }
        r1 = make_float2(f32_of((double)rho1.x), f32_of((double)rho1.y));
      }
      for (int m = Mh; m < M; ++m) {
        const float2 w0 = make_float2(f0 * c0.x, f0 * c0.y);
        const float2 w1 = make_float2(f1 * c1.x, -f1 * c1.y);
        for (int s = 0; s < B.K; ++s) {
          float2* u = U32 + (int64_t)(s * Ml + m - Mh) * N;
          u[kp] = (s == s0) ? w0 : make_float2(0.f, 0.f);
          u[N - 1 - kp] = (s == s1) ? w1 : make_float2(0.f, 0.f);
        }
        if (m + 1 < M) {
          const float p0 = pow2f(g0[m + 1] - g0[m]), p1 = pow2f(g1[m + 1] - g1[m]);
          c0 = cmulf(c0, make_float2(r0.x * p0, r0.y * p0));
          c1 = cmulf(c1, make_float2(r1.x * p1, r1.y * p1));
        }
      }
    }
  }
}

// With F the T2-type transform of band s, term m, the DCT-II part minus the
// DST-II part of the pair, (e.x (Fn.x + Fm.x) + e.y (Fn.y - Fm.y)) +
// (e.x (Fm.x - Fn.x) - e.y (Fm.y + Fn.y)), is 2 Re(e_n F_{N-n}) (and 2 Re F_0 at
// n = 0, where e = 1): only the bin N - n is read, and the sum over bands and
// terms is taken before the rotation,
//   out_n = rect_n + Re(e_n sum_m C_n h_{m,n} sum_{s: n >= n_s} F^{(s,m)}_{N-n}).
template <typename T>
__global__ void k_l2ct_epi(const C2<T>* __restrict__ F, const ffc* __restrict__ Fff,
                           const float2* __restrict__ F32, const T* __restrict__ rect, T* __restrict__ out, int64_t N,
                           int M, int Mh, int M64, BandArgs B, const double* __restrict__ Cn,
                           const double* __restrict__ Hnm, int scale_s, TwArgs<T> tw4N, Scale32 S,
                           const double* __restrict__ hb, int64_t hh, int64_t hs) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t bt = blockIdx.y;
  const int Ml = M - Mh, Mf = Mh - M64;
  rect += bt * N;
  out += bt * N;
  if (F) F += bt * (int64_t)B.K * M64 * N;
  if (Fff) Fff += bt * (int64_t)B.K * Mf * N;
  if (F32) F32 += bt * (int64_t)B.K * Ml * N;
  T acc = rect[n];
  if (B.K > 0 && M > 0) {
    const int64_t nm = (N - n) & (N - 1);
    int s0 = 0;  // bands s >= s0 have n >= n_s (the cuts decrease with s)
    while (s0 < B.K && n < B.ns[s0]) ++s0;
    if (s0 < B.K) {
      HTerm<T> H{Hnm, N, n, sizeof(T) == 8 ? (T)0 : (T)Cn[n], (T)1};
      C2<T> V = mk<T>((T)0, (T)0);
      for (int m = 0; m < M64; ++m) {
        C2<T> X = F[(int64_t)(s0 * M64 + m) * N + nm];
        for (int s = s0 + 1; s < B.K; ++s) X = cadd<T>(X, F[(int64_t)(s * M64 + m) * N + nm]);
        const T hm = H.at(m);
        V = mk<T>(V.x + hm * X.x, V.y + hm * X.y);
      }
      if (Mf > 0) {
        // float-float terms: band s's output is scaled by 2^{g_{s,m} - E}; with
        // Hff = C_n h_{m,n} 2^{e_{K-1,m}} the term is
        // 2^E Hff sum_s 2^{-e_{K-1,m} - g_{s,m}} Fff, summed in float-float
        const int* eK = S.e + (B.K - 1) * M;
        const int* et = S.e + B.K * M;
        ffd vx(0.f, 0.f), vy(0.f, 0.f);
        for (int m = M64; m < Mh; ++m) {
          ffd xx(0.f, 0.f), xy(0.f, 0.f);
          for (int s = s0; s < B.K; ++s) {
            const ffc q = Fff[(int64_t)(s * Mf + m - M64) * N + nm];
            const float p = pow2f(-eK[m] - et[s * M + m]);
            xx = xx + ffd(q.x.hi * p, q.x.lo * p);
            xy = xy + ffd(q.y.hi * p, q.y.lo * p);
          }
          const ffd h = S.Hff[(int64_t)(m - M64) * N + n];
          vx = vx + h * xx;
          vy = vy + h * xy;
        }
        const int E = item_exp(S, bt);
        V = mk<T>(V.x + (T)scale2(dbl_of(vx), E), V.y + (T)scale2(dbl_of(vy), E));
      }
      if (Ml > 0) {
        // FP32 terms: band s's output is scaled by 2^{g_{s,m} - E}; with
        // H32 = C_n h_{m,n} 2^{e_{K-1,m}} the term is 2^E H32 sum_s 2^{-e_{K-1,m} - g_{s,m}} F32
        const int* eK = S.e + (B.K - 1) * M;
        const int* et = S.e + B.K * M;
        float vx = 0.f, vy = 0.f;
        for (int m = Mh; m < M; ++m) {
          float xx = 0.f, xy = 0.f;
          for (int s = s0; s < B.K; ++s) {
            const float2 q = F32[(int64_t)(s * Ml + m - Mh) * N + nm];
            const float p = pow2f(-eK[m] - et[s * M + m]);
            xx = fmaf(p, q.x, xx);
            xy = fmaf(p, q.y, xy);
          }
          const float h32 = S.H32[(int64_t)(m - Mh) * N + n];
          vx = fmaf(h32, xx, vx);
          vy = fmaf(h32, xy, vy);
        }
        const int E = item_exp(S, bt);
        V = mk<T>(V.x + (T)scale2(f64_of(vx), E), V.y + (T)scale2(f64_of(vy), E));
      }
      const C2<T> e = twid<T>(tw4N, n);
      acc += e.x * V.x - e.y * V.y;
    }
  }
  const T val = scale_s ? (idx_t<T>(n) + (T)0.5) * acc : acc;
  // the head block's columns (when it ran beside this chain): added in double
  out[n] = (hb && n < hh) ? (T)((double)val + hb[bt * hs + n]) : val;
}

// which: 0 copy, 1 multiply by (n + 1/2), 2 multiply by w_k, 3 dtheta = tN / N (double out)
template <typename T>
__global__ void k_scale(const T* __restrict__ in, T* __restrict__ out, const double* __restrict__ w,
                        int64_t N, int which) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  in += (int64_t)blockIdx.y * N;
  out += (int64_t)blockIdx.y * N;
  T v = in[n];
  if (which == 1) v *= (idx_t<T>(n) + (T)0.5);
  if (which == 2) v *= (T)w[n];
  out[n] = v;
}

constexpr int TPB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

Scale32 scale32(const Plan& P) { return Scale32{P.b32exp, P.absmax, P.H32, P.Hff}; }

// amax[item] = max over n of |x_n| as the bits of a non-negative double (their
// integer order is the order of the values); amax is zeroed before the launch
template <typename T>
__global__ void k_absmax(const T* __restrict__ x, int64_t N, unsigned long long* __restrict__ amax) {
  x += (int64_t)blockIdx.y * N;
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)x[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(amax + blockIdx.y, (unsigned long long)__double_as_longlong(m));
}

}  // namespace

template <typename T>
int launch_l2c_pro(Plan& P, const T* c, C2<T>* U, ffc* Uff, float2* U32, int64_t nb) {
  const TwArgs<T> tw = tw4n_args<T>(P);
  k_l2c_pro<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(
      c, U, Uff, U32, P.p.N, P.p.M, P.p.Mh, P.p.M64, band_args(P), P.Cn, P.Hnm, tw, scale32(P));
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "l2c_pro", (double)nb * (10.0 * P.p.M * N), (double)nb * (ts * N + 8.0 * N + KM * N * cs));
  }
  return check_launch();
}
template <typename T>
int launch_l2c_epi(Plan& P, const C2<T>* Y, const ffc* Yff, const float2* Y32, const T* vrec, T* v, int64_t nb) {
  k_l2c_epi<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(
      Y, Yff, Y32, vrec, v, P.p.N, P.p.M, P.p.Mh, P.p.M64, band_args(P), P.row_ar, scale32(P));
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "l2c_epi", (double)nb * (10.0 * P.p.M * N), (double)nb * (P.p.M * N * cs + 2.0 * ts * N));
  }
  return check_launch();
}
template <typename T>
int launch_a4_pro(Plan& P, const T* v, C2<T>* U, int64_t nb) {
  k_a4_pro<T><<<dim3(nblk(P.p.N / 2), (unsigned)nb), TPB, 0, P.stream>>>(v, U, P.p.N);
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "a4_pro", (double)nb * (0.0), (double)nb * (ts * N + N * cs));
  }
  return check_launch();
}
template <typename T>
int launch_a4_epi(Plan& P, const C2<T>* F, T* chat, int64_t nb, const double* hb) {
  const TwArgs<T> tw = tw4n_args<T>(P);
  k_a4_epi<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(F, chat, P.p.N, (T)1 / (T)P.p.N, tw, hb,
                                                                     P.p.head, P.p.N * (int64_t)sizeof(T) / 8);
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "a4_epi", (double)nb * (12.0 * N), (double)nb * (2.0 * N * cs + ts * N));
  }
  return check_launch();
}
template <typename T>
int launch_fcs_pro(Plan& P, const T* a, C2<T>* U, int scale_d, int64_t nb) {
  const TwArgs<T> tw = tw4n_args<T>(P);
  k_fcs_pro<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(a, U, P.p.N, scale_d, (T)1 / (T)P.p.N, tw);
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "fcs_pro", (double)nb * (8.0 * N), (double)nb * (ts * N + N * cs));
  }
  return check_launch();
}
template <typename T>
int launch_fcs_re_epi(Plan& P, const C2<T>* Y, T* out, int64_t nb) {
  k_fcs_re_epi<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(Y, out, P.p.N);
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "fcs_re_epi", (double)nb * (0.0), (double)nb * (N * cs + ts * N));
  }
  return check_launch();
}
template <typename T>
int launch_tay_pro(Plan& P, const T* chat, C2<T>* U, ffc* Uff, int inc0, int npair, int64_t nb) {
  const TwArgs<T> tw = tw4n_args<T>(P);
  const int P64 = Uff ? taylor_p64(P.p, inc0, npair) : npair;
  k_tay_pro<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(chat, U, Uff, P.p.N, P.p.L, inc0, npair, P64,
                                                                       (T)1 / (T)P.p.N, tw, scale32(P));
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "tay_pro", (double)nb * (16.0 * npair * N), (double)nb * (2.0 * ts * N + npair * N * cs));
  }
  return check_launch();
}
template <typename T>
int launch_tay_epi(Plan& P, const C2<T>* Y, const ffc* Yff, const T* v, T* f, int inc0, int npair, int64_t nb) {
  const int P64 = Yff ? taylor_p64(P.p, inc0, npair) : npair;
  if (int st = nodes_ready(P)) return st;
  if (P.rg_rules)
    k_tay_epi<T, true><<<dim3(nblk(P.rg_nmax), (unsigned)nb), TPB, 0, P.stream>>>(
        Y, Yff, v, f, nullptr, P.p.N, P.p.L, inc0, npair, P64, scale32(P), P.rg_rules,
        P.rg_item ? P.rg_item + P.rg_item0 : nullptr);
  else
    k_tay_epi<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(Y, Yff, v, f, P.tN, P.p.N, P.p.L, inc0,
                                                                         npair, P64, scale32(P));
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "tay_epi", (double)nb * ((2.0 * P.p.L + 6.0 * npair) * N), (double)nb * (npair * N * cs + 2.0 * ts * N + 8.0 * N));
  }
  return check_launch();
}
template <typename T>
int launch_tayt_pro(Plan& P, const T* f, int use_w, C2<T>* U, ffc* Uff, int inc0, int npair, int64_t nb) {
  const int P64 = Uff ? taylor_p64(P.p, inc0, npair) : npair;
  if (int st = nodes_ready(P)) return st;
  if (P.rg_rules)
    k_tayt_pro_grid<T><<<dim3(nblk(P.p.N / 2), (unsigned)nb), TPB, 0, P.stream>>>(
        f, use_w, P.rg_rules, P.rg_item ? P.rg_item + P.rg_item0 : nullptr, U, Uff, P.p.N, P.p.L, inc0, npair, P64,
        scale32(P));
  else
    k_tayt_pro<T><<<dim3(nblk(P.p.N / 2), (unsigned)nb), TPB, 0, P.stream>>>(f, use_w ? P.w : nullptr, P.tN, U, Uff,
                                                                             P.p.N, P.p.L, inc0, npair, P64,
                                                                             scale32(P));
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "tayt_pro", (double)nb * (8.0 * npair * N), (double)nb * (ts * N + 16.0 * N + npair * N * cs));
  }
  return check_launch();
}
template <typename T>
int launch_tayt_epi(Plan& P, const C2<T>* F, const ffc* Fff, C2<T>* Q, T* u_out, int inc0, int npair, int64_t nb,
                    int64_t nu) {
  const TwArgs<T> tw = tw4n_args<T>(P);
  if (nu < 0) nu = P.p.N;
  const int P64 = Fff ? taylor_p64(P.p, inc0, npair) : npair;
  k_tayt_epi<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(F, Fff, Q, u_out, P.p.N, P.p.L, inc0, npair,
                                                                        P64, nu, (T)1 / (T)P.p.N, tw, scale32(P));
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "tayt_epi", (double)nb * ((2.0 * P.p.L + 16.0 * npair) * N), (double)nb * (2.0 * npair * N * cs + N * cs));
  }
  return check_launch();
}
template <typename T>
int launch_l2ct_pro(Plan& P, const C2<T>* Y, const T* g, int use_w, T* z, C2<T>* U, ffc* Uff, float2* U32,
                    int64_t nb) {
  const double* w = use_w ? P.w : nullptr;
  k_l2ct_pro<T><<<dim3(nblk(P.p.N / 2), (unsigned)nb), TPB, 0, P.stream>>>(
      Y, g, w, z, U, Uff, U32, P.p.N, P.p.M, P.p.Mh, P.p.M64, band_args(P), P.row_ar, scale32(P));
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "l2ct_pro", (double)nb * (10.0 * P.p.M * N), (double)nb * (N * cs + 2.0 * ts * N + 8.0 * N + KM * N * cs));
  }
  return check_launch();
}
template <typename T>
int launch_l2ct_epi(Plan& P, const C2<T>* F, const ffc* Fff, const float2* F32, const T* rect, T* out, int scale_s,
                    int64_t nb, const double* hb) {
  const TwArgs<T> tw = tw4n_args<T>(P);
  k_l2ct_epi<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(
      F, Fff, F32, rect, out, P.p.N, P.p.M, P.p.Mh, P.p.M64, band_args(P), P.Cn, P.Hnm, scale_s, tw, scale32(P), hb,
      P.p.head, P.p.N * (int64_t)sizeof(T) / 8);
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "l2ct_epi", (double)nb * (4.0 * KM * N), (double)nb * (KM * N * cs + 2.0 * ts * N));
  }
  return check_launch();
}
template <typename T>
int launch_absmax(Plan& P, const T* x, int64_t nb) {
  if (!P.absmax) return GBDLT_OK;
  if (cudaMemsetAsync(P.absmax, 0, sizeof(unsigned long long) * (size_t)nb, P.stream) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  const int64_t blocks = std::min<int64_t>(nblk(P.p.N), 2 * 152);
  k_absmax<T><<<dim3((unsigned)blocks, (unsigned)nb), TPB, 0, P.stream>>>(x, P.p.N, P.absmax);
  launched(P, "absmax", (double)nb * P.p.N, (double)nb * sizeof(T) * P.p.N);
  return check_launch();
}
template <typename T>
int launch_scale(Plan& P, const T* in, T* out, int which, int64_t nb) {
  if (which == 2)
    if (int st = nodes_ready(P)) return st;  // the weights
  k_scale<T><<<dim3(nblk(P.p.N), (unsigned)nb), TPB, 0, P.stream>>>(in, out, P.w, P.p.N, which);
  {
    const double N = (double)P.p.N, ts = sizeof(T), cs = 2.0 * sizeof(T);
    const double KM = (double)P.p.K * P.p.M;
    (void)KM;
    launched(P, "scale", (double)nb * (N), (double)nb * (2.0 * ts * N + 8.0 * N));
  }
  return check_launch();
}

int launch_stage_tables_init(Plan& P) {
  const int64_t N = P.p.N;
  if (P.row_ar) {
    k_row_factors_init<<<nblk(N), TPB, 0, P.stream>>>(P.row_ar, N);
    count_launch();
  }
  if (P.Hnm) {
    // entries of the float-float and FP32 terms only with their tables
    const int Mh = P.Hff ? P.p.Mh : P.p.M64;
    const int Mt = P.H32 ? P.p.M : Mh;
    const int* eK = P.b32exp ? P.b32exp + (P.p.K - 1) * P.p.M : nullptr;
    const int64_t ns_min = P.p.K > 0 ? P.p.bands[(size_t)P.p.K - 1].ns : N;
    k_hnm_init<<<nblk(N), TPB, 0, P.stream>>>(P.Hnm, P.Hff, P.H32, P.Cn, N, Mt, Mh, P.p.M64, eK, ns_min);
    count_launch();
  }
  return check_launch();
}

#define INST(T)                                                                              \
  template int launch_l2c_pro<T>(Plan&, const T*, C2<T>*, ffc*, float2*, int64_t);                    \
  template int launch_absmax<T>(Plan&, const T*, int64_t);                                            \
  template int launch_l2c_epi<T>(Plan&, const C2<T>*, const ffc*, const float2*, const T*, T*, int64_t); \
  template int launch_a4_pro<T>(Plan&, const T*, C2<T>*, int64_t);                                    \
  template int launch_a4_epi<T>(Plan&, const C2<T>*, T*, int64_t, const double*);                     \
  template int launch_fcs_pro<T>(Plan&, const T*, C2<T>*, int, int64_t);                              \
  template int launch_fcs_re_epi<T>(Plan&, const C2<T>*, T*, int64_t);                                \
  template int launch_tay_pro<T>(Plan&, const T*, C2<T>*, ffc*, int, int, int64_t);                   \
  template int launch_tay_epi<T>(Plan&, const C2<T>*, const ffc*, const T*, T*, int, int, int64_t);   \
  template int launch_tayt_pro<T>(Plan&, const T*, int, C2<T>*, ffc*, int, int, int64_t);             \
  template int launch_tayt_epi<T>(Plan&, const C2<T>*, const ffc*, C2<T>*, T*, int, int, int64_t, int64_t); \
  template int launch_l2ct_pro<T>(Plan&, const C2<T>*, const T*, int, T*, C2<T>*, ffc*, float2*, int64_t); \
  template int launch_l2ct_epi<T>(Plan&, const C2<T>*, const ffc*, const float2*, const T*, T*, int, int64_t, \
                                  const double*);                                                      \
  template int launch_scale<T>(Plan&, const T*, T*, int, int64_t);
INST(double)
INST(float)
#undef INST

}  // namespace gbdlt
