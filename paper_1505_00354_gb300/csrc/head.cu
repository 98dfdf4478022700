// Dense head block of leg2cheb (Sec. 3, the matrix M with chat = M c) and of its
// transpose.  The first h Legendre columns map to the first h Chebyshev
// coefficients only (M is upper triangular), through
//   M_{0n} = Lam'_{n/2}^2 / 2,   M_{kn} = Lam'_{(n-k)/2} Lam'_{(n+k)/2}   (0 < k <= n, n - k even),
// with Lam'_j = sqrt(2/pi) Gamma(j+1/2)/Gamma(j+1) (the plan's table, computed
// in double-double on the host).  A fast plan with head h takes columns n < h
// from this block, so no asymptotic band cuts below h and every recurrence row
// starts at n = h.
//   forward     chat_k += sum_{j : k+2j < h} Lam'_j Lam'_{j+k} c_{k+2j}       (halved at k = 0)
//   transposed  out_n  += s_n sum_{j <= n/2} Lam'_j Lam'_{n-j} y_{n-2j}      (halved where n = 2j),
//               s_n = n + 1/2 when the chain scales its output, else 1.
// One warp per output: lanes stride over j, so the table and input reads of a
// warp are contiguous; the sum is a plain FP64 fused multiply-add chain in the
// FP64 form and a Kahan-compensated FP32 sum in the FP32 form (FP32 arithmetic
// runs on a pipe 64 times wider than FP64 on GB300).  Per term: one product of
// two table entries and one multiply-add, so FP64 issue bounds the FP64 form;
// FP64 plans with h <= kHeadTabMax use the stored products below instead.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "gbdlt_internal.cuh"

namespace gbdlt {

namespace {

constexpr int HW = 8;  // warps (outputs) per CTA

__device__ __forceinline__ void kahan_acc(float& s, float& c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// sum over lanes of a lane partial, in double
__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// lane partial of sum_{j in [0, J), j = lane mod 32} lam[a0 + j] lam[b0 + s_b j] x[x0 + s_x j]
template <typename T>
struct HeadSum;

template <>
struct HeadSum<double> {
  __device__ __forceinline__ static double run(const double* __restrict__ lam, const double* __restrict__ x,
                                               int64_t b0, int sb, int64_t x0, int sx, int64_t J, int lane) {
    double a0 = 0.0, a1 = 0.0;
    int64_t j = lane;
    for (; j + 32 < J; j += 64) {
      a0 = fma(lam[j] * lam[b0 + sb * j], x[x0 + sx * j], a0);
      const int64_t j2 = j + 32;
      a1 = fma(lam[j2] * lam[b0 + sb * j2], x[x0 + sx * j2], a1);
    }
    if (j < J) a0 = fma(lam[j] * lam[b0 + sb * j], x[x0 + sx * j], a0);
    return a0 + a1;
  }
};

template <>
struct HeadSum<float> {
  __device__ __forceinline__ static double run(const float* __restrict__ lam, const float* __restrict__ x,
                                               int64_t b0, int sb, int64_t x0, int sx, int64_t J, int lane) {
    float s = 0.f, c = 0.f;
    for (int64_t j = lane; j < J; j += 32) kahan_acc(s, c, lam[j] * lam[b0 + sb * j] * x[x0 + sx * j]);
    return (double)s - (double)c;
  }
};

// hout != null: the block's sum goes to hout[k] (double, item stride hs) instead
// of being added to chat (the chain adds it in the A4 epilogue)
template <typename T>
__global__ void __launch_bounds__(HW * 32) k_head_fwd(const T* __restrict__ c, T* __restrict__ chat,
                                                      const T* __restrict__ lam, int64_t N, int64_t h,
                                                      double* __restrict__ hout, int64_t hs) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * HW + (threadIdx.x >> 5);
  if (k >= h) return;  // whole warp
  c += (int64_t)blockIdx.y * N;
  chat += (int64_t)blockIdx.y * N;
  const int64_t J = (h - k + 1) / 2;  // j < J  <=>  k + 2j < h
  // term j: lam[j] lam[k + j] c[k + 2j]
  double s = warp_sum(HeadSum<T>::run(lam, c, k, 1, k, 2, J, lane));
  if (k == 0) s *= 0.5;
  if (lane == 0) {
    if (hout)
      hout[(int64_t)blockIdx.y * hs + k] = s;
    else
      chat[k] = (T)((double)chat[k] + s);
  }
}

// hout != null: the scaled sum goes to hout[n] (double, item stride hs) instead of
// being added to out (the chain adds it in the transposed leg2cheb epilogue)
template <typename T>
__global__ void __launch_bounds__(HW * 32) k_head_t(const T* __restrict__ y, T* __restrict__ out,
                                                    const T* __restrict__ lam, int64_t N, int64_t h, int scale_s,
                                                    double* __restrict__ hout, int64_t hs) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * HW + (threadIdx.x >> 5);
  if (q >= h) return;  // whole warp
  const int64_t n = h - 1 - q;  // longest sums first
  y += (int64_t)blockIdx.y * N;
  out += (int64_t)blockIdx.y * N;
  // terms j with n - 2j > 0 in the loop; the k = 0 term (n even) halved after it
  const int64_t J = (n + 1) / 2;
  // term j: lam[j] lam[n - j] y[n - 2j]
  double s = warp_sum(HeadSum<T>::run(lam, y, n, -1, n, -2, J, lane));
  if (lane == 0) {
    if (!(n & 1)) s += 0.5 * (double)lam[n / 2] * (double)lam[n / 2] * (double)y[0];
    if (scale_s) s *= (double)n + 0.5;
    if (hout)
      hout[(int64_t)blockIdx.y * hs + n] = s;
    else
      out[n] = (T)((double)out[n] + s);
  }
}

// ---------------------------------------------------------------- stored products
// FP64 plans with h <= kHeadTabMax keep the products M_{k,n} = Lam'_j Lam'_{j+k}
// (n = k + 2j) in a table, row k holding n = k, k+2, ..., < h from offset off[k]
// (h^2/4 doubles: 537 MB at h = 16384).  Each term then costs one FP64 fused
// multiply-add and 8 bytes of HBM instead of a product and a fused multiply-add:
// the FP64 work halves, and the table streams from HBM at about 4 TB/s beside
// it.  The stored product is the rounded product the on-the-fly kernel forms, so
// the forward block is bitwise the same.
__global__ void k_head_tab_init(const double* __restrict__ lam, const int64_t* __restrict__ off,
                                double* __restrict__ tab, int64_t h) {
  const int64_t k = blockIdx.x;
  const int64_t J = (h - k + 1) / 2;
  double* row = tab + off[k];
  for (int64_t j = threadIdx.x; j < J; j += blockDim.x) row[j] = lam[j] * lam[k + j];
}

// column n of the transposed table: entry i is row k = (n mod 2) + 2i, the
// product Lam'_{(n-k)/2} Lam'_{(n+k)/2} rounded as in the row table
__global__ void k_head_tabT_init(const double* __restrict__ lam, const int64_t* __restrict__ offT,
                                 double* __restrict__ tabT, int64_t h) {
  const int64_t n = blockIdx.x;
  const int64_t p = n & 1;
  const int64_t I = (n - p) / 2 + 1;
  double* col = tabT + offT[n];
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
    const int64_t k = p + 2 * i;
    const int64_t j = (n - k) / 2;
    col[i] = lam[j] * lam[j + k];
  }
}

// transposed from the column table: one warp per output n (longest columns
// first), lanes over the rows, the row-0 term halved
__global__ void __launch_bounds__(HW * 32) k_head_t_tabT(const double* __restrict__ y, double* __restrict__ out,
                                                         const double* __restrict__ tabT,
                                                         const int64_t* __restrict__ offT, int64_t N, int64_t h,
                                                         int scale_s, double* __restrict__ hout, int64_t hs) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * HW + (threadIdx.x >> 5);
  if (q >= h) return;  // whole warp
  const int64_t n = h - 1 - q;
  const int64_t p = n & 1;
  y += (int64_t)blockIdx.y * N;
  out += (int64_t)blockIdx.y * N;
  const int64_t I = (n - p) / 2 + 1;
  const double* __restrict__ col = tabT + offT[n];
  const double* __restrict__ x = y + p;
  double a0 = 0.0, a1 = 0.0;
  int64_t i = lane;
#pragma unroll 4
  for (; i + 32 < I; i += 64) {
    a0 = fma(col[i], x[2 * i], a0);
    a1 = fma(col[i + 32], x[2 * (i + 32)], a1);
  }
  if (i < I) a0 = fma(col[i], x[2 * i], a0);
  double s = a0 + a1;
  // the row k = 0 term (even n) enters halved: lane 0 took it in full
  if (p == 0 && lane == 0) s = fma(-0.5 * col[0], y[0], s);
  s = warp_sum(s);
  if (lane == 0) {
    if (scale_s) s *= (double)n + 0.5;
    if (hout)
      hout[(int64_t)blockIdx.y * hs + n] = s;
    else
      out[n] = out[n] + s;
  }
}

// forward: one warp per output k, lanes over j (the on-the-fly kernel's order)
__global__ void __launch_bounds__(HW * 32) k_head_fwd_tab(const double* __restrict__ c, double* __restrict__ chat,
                                                          const double* __restrict__ tab,
                                                          const int64_t* __restrict__ off, int64_t N, int64_t h) {
  const int lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * HW + (threadIdx.x >> 5);
  if (k >= h) return;  // whole warp
  c += (int64_t)blockIdx.y * N;
  chat += (int64_t)blockIdx.y * N;
  const int64_t J = (h - k + 1) / 2;
  const double* __restrict__ row = tab + off[k];
  const double* __restrict__ x = c + k;
  double a0 = 0.0, a1 = 0.0;
  int64_t j = lane;
#pragma unroll 4
  for (; j + 32 < J; j += 64) {
    a0 = fma(row[j], x[2 * j], a0);
    a1 = fma(row[j + 32], x[2 * (j + 32)], a1);
  }
  if (j < J) a0 = fma(row[j], x[2 * j], a0);
  double s = warp_sum(a0 + a1);
  if (k == 0) s *= 0.5;
  if (lane == 0) chat[k] = chat[k] + s;
}

// transposed: a CTA takes 32 columns n = 64 g + par + 2 lane of one parity and its
// TW warps split the rows k = par, par + 2, ... <= n among them (row k's entry for
// column n sits at off[k] + (n - k)/2, so a warp's loads are contiguous); the
// row k = 0 term is halved; the warps' partial sums are added in shared memory
constexpr int TW = 16;
__global__ void __launch_bounds__(TW * 32) k_head_t_tab(const double* __restrict__ y, double* __restrict__ out,
                                                        const double* __restrict__ tab,
                                                        const int64_t* __restrict__ off, int64_t N, int64_t h,
                                                        int scale_s, double* __restrict__ hout, int64_t hs) {
  __shared__ double red[TW][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t ng = (h + 63) / 64;
  const int64_t g = ng - 1 - (int64_t)(blockIdx.x >> 1);  // longest sums first
  const int par = blockIdx.x & 1;
  const int64_t n = 64 * g + par + 2 * lane;
  y += (int64_t)blockIdx.y * N;
  out += (int64_t)blockIdx.y * N;
  const int64_t R = 32 * g + 32;  // rows k = par + 2 i, i < R, cover k <= 64 g + par + 62
  const int64_t i0 = (int64_t)w * R / TW, i1 = (int64_t)(w + 1) * R / TW;
  // batches of 8 rows: their 8 (independent) loads are in flight together
  constexpr int B8 = 8;
  const double y0h = 0.5 * y[0];  // the row k = 0 term is halved
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t ib = i0; ib < i1; ib += B8) {
    double m[B8], yv[B8];
#pragma unroll
    for (int q = 0; q < B8; ++q) {
      const int64_t i = ib + q;
      const int64_t k = par + 2 * i;
      const bool live = i < i1 && n < h && k <= n;
      m[q] = live ? tab[off[k] + ((n - k) >> 1)] : 0.0;
      yv[q] = live ? (k == 0 ? y0h : y[k]) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < B8; ++q) a[q & 3] = fma(m[q], yv[q], a[q & 3]);
  }
  const double a0 = a[0] + a[1], a1 = a[2] + a[3];
  red[w][lane] = a0 + a1;
  __syncthreads();
  if (w == 0 && n < h) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < TW; ++q) s += red[q][lane];
    if (scale_s) s *= (double)n + 0.5;
    if (hout)
      hout[(int64_t)blockIdx.y * hs + n] = s;
    else
      out[n] = out[n] + s;
  }
}

// ---------------------------------------------------------------- tiled product (h <= kHeadMM)
// FP32 plans with a small head block (h <= kHeadMM, N <= 8192) run both
// directions as one tiled product over the batch, for single and batched calls
// alike (FP64 plans keep the per-warp kernels with stored products, which
// measured faster: 0.26 against 0.31 ms for 246 items at N = 4096).  Per
// parity p the block is G_p[a][m] = Lam'_{m-a} Lam'_{m+a+p} (a <= m, halved at
// a = 0 when p = 0; a exact power-of-two scaling), k = p + 2a, n = p + 2m:
//   forward     chat_{p+2a} += sum_{m >= a} G_p[a][m] c_{p+2m}
//   transposed  out_{p+2m}  += s_n sum_{a <= m} G_p[a][m] y_{p+2a}.
// A CTA computes 64 outputs of one parity for 32 batch items; the reduction
// index runs through chunks of 32 staged in shared memory (G entries formed
// there from the table, the inputs gathered), and each output is summed in
// ascending reduction order, sequentially (an FP64 fused multiply-add chain, a
// Kahan-compensated FP32 sum), so the result of an item does not depend on how
// many items a call carries.  Thread t: item t mod 32, outputs 8 (t / 32) + i.
constexpr int MMO = 64, MMB = 32, MMR = 32;

template <typename T, bool TRANS>
__global__ void __launch_bounds__(256) k_head_mm(const T* __restrict__ x, T* __restrict__ out,
                                                 const T* __restrict__ lam, int64_t N, int64_t h, int scale_s,
                                                 double* __restrict__ hout, int64_t hs, int64_t nb) {
  __shared__ T Gs[MMR][MMO];
  __shared__ T Xs[MMR][MMB];
  const int par = blockIdx.x & 1;
  const int64_t H = (h - par + 1) / 2;  // indices of this parity below h
  const int64_t o0 = (int64_t)(blockIdx.x >> 1) * MMO;
  const int64_t b0 = (int64_t)blockIdx.y * MMB;
  if (o0 >= H) return;  // whole CTA
  const int tb = threadIdx.x & 31, og = threadIdx.x >> 5;
  // reduction range: forward r = m in [o0, H), transposed r = a in [0, min(o0 + MMO, H))
  const int64_t r_lo = TRANS ? 0 : o0;
  const int64_t r_hi = TRANS ? min(o0 + MMO, H) : H;
  T acc[8], cmp[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = cmp[i] = (T)0;
  for (int64_t r0 = r_lo; r0 < r_hi; r0 += MMR) {
    // G tile: entry (rr, oo) for reduction index r0 + rr and output o0 + oo
    for (int e = threadIdx.x; e < MMR * MMO; e += 256) {
      const int rr = e / MMO, oo = e % MMO;
      const int64_t r = r0 + rr, o = o0 + oo;
      const int64_t a = TRANS ? r : o, m = TRANS ? o : r;
      T g = (T)0;
      if (r < r_hi && o < H && a <= m) {
        g = lam[m - a] * lam[m + a + par];
        if (par == 0 && a == 0) g *= (T)0.5;
      }
      Gs[rr][oo] = g;
    }
    for (int e = threadIdx.x; e < MMR * MMB; e += 256) {
      const int rr = e / MMB, bb = e % MMB;
      const int64_t r = r0 + rr, b = b0 + bb;
      Xs[rr][bb] = (r < r_hi && b < nb) ? x[b * N + par + 2 * r] : (T)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < MMR; ++rr) {
      const T xv = Xs[rr][tb];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const T g = Gs[rr][og * 8 + i];
        if constexpr (std::is_same<T, double>::value) {
          acc[i] = fma(g, xv, acc[i]);
        } else {
          // Kahan step on the product g x (the per-warp kernels' arithmetic)
          const float v = __fmul_rn(g, xv);
          const float y = __fsub_rn(v, cmp[i]);
          const float t = __fadd_rn(acc[i], y);
          cmp[i] = __fsub_rn(__fsub_rn(t, acc[i]), y);
          acc[i] = t;
        }
      }
    }
    __syncthreads();
  }
  const int64_t b = b0 + tb;
  if (b >= nb) return;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t o = o0 + og * 8 + i;
    if (o >= H) break;
    const int64_t idx = par + 2 * o;  // output coefficient k (forward) or n (transposed)
    double s = std::is_same<T, double>::value ? (double)acc[i] : (double)acc[i] - (double)cmp[i];
    if (TRANS && scale_s) s *= (double)idx + 0.5;
    if (hout)
      hout[b * hs + idx] = s;
    else
      out[b * N + idx] = (T)((double)out[b * N + idx] + s);
  }
}

// ---------------------------------------------------------------- FP32, register-blocked (h > kHeadMM)
// Per parity p the block is G_p[a][m] = Lam'_{m-a} Lam'_{m+a+p} (a <= m; k = p + 2a,
// n = p + 2m).  A warp task takes 256 consecutive outputs of one parity (8 per
// lane: o_i = o0 + i) and one chunk of rbc reduction indices r (a multiple of 8
// chosen per plan, head_rb_tasks):
//   forward     out a = o_i, reduction m = r:  term Lam'[r - o_i] Lam'[r + o_i + p] x_{p+2r}
//   transposed  out m = o_i, reduction a = r:  term Lam'[o_i - r] Lam'[o_i + r + p] y_{p+2r}
// (y_0 halved for p = 0).  From one r to the next the first factors of a lane's
// 8 outputs move up one output and the second ones down one, so the entry a
// lane needs next is held by its neighbour lane (a warp shuffle) and the warp
// loads only the two entries entering at its edges and the input x_{p+2r}, each
// one address for all lanes; terms outside the triangle read the table's zero
// padding (index below 0) and vanish.  Each output sums its terms 8 at a time in
// FP32 fused multiply-adds and those block sums in a Kahan-compensated FP32 sum
// in ascending r; k_head_rb_reduce adds the chunk sums of an output in ascending
// chunk order in double.
constexpr int RB = 8;
constexpr int RBW = 32 * RB;

template <bool TRANS>
__global__ void __launch_bounds__(256) k_head_rb(const float* __restrict__ x, const float* __restrict__ lamp,
                                                 const int4* __restrict__ tasks, int ntask, int64_t N, int64_t h,
                                                 int rbc, double* __restrict__ part, int64_t part_n) {
  const int task = (int)blockIdx.x * 8 + (int)(threadIdx.x >> 5);
  if (task >= ntask) return;  // whole warp
  const int4 tk = tasks[task];
  const int par = tk.x;
  const int lane = threadIdx.x & 31;
  const int64_t Hp = (h - par + 1) / 2;
  const int64_t H0 = (h + 1) / 2;
  const int64_t nch = (H0 + rbc - 1) / rbc;
  x += (int64_t)blockIdx.y * N;
  const float* __restrict__ lam = lamp + kHeadPad;
  const int64_t oB = (int64_t)tk.y * RBW;
  const int64_t o0 = oB + lane * RB;
  const int64_t r0 = (int64_t)tk.z * rbc;
  const int64_t rend = TRANS ? min(Hp, (int64_t)(tk.y + 1) * RBW) : Hp;
  const int64_t r1 = min(r0 + rbc, rend);
  // T[i] = Lam'[r - o_i] (forward) or Lam'[o_i - r] (transposed), H[i] = Lam'[r + o_i + p]
  float T[RB], H[RB], acc[RB], cmp[RB];
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    T[i] = lam[TRANS ? (o0 + i - r0) : (r0 - o0 - i)];
    H[i] = lam[r0 + o0 + i + par];
    acc[i] = cmp[i] = 0.f;
  }
  for (int64_t R = r0; R < r1; R += RB) {
    // the entries that enter at the warp's edges over the next RB steps (one
    // address per load for the whole warp), and the inputs
    float tl[RB], hl[RB], xv[RB];
#pragma unroll
    for (int st = 0; st < RB; ++st) {
      const int64_t r = R + st;
      tl[st] = lam[TRANS ? (oB - r - 1) : (r + 1 - oB)];
      hl[st] = lam[r + 1 + oB + RBW - 1 + par];
      float v = r < r1 ? x[par + 2 * r] : 0.f;
      if (TRANS && par == 0 && r == 0) v *= 0.5f;
      xv[st] = v;
    }
    float b[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) b[i] = 0.f;
#pragma unroll
    for (int st = 0; st < RB; ++st) {
#pragma unroll
      for (int i = 0; i < RB; ++i) b[i] = fmaf(__fmul_rn(T[i], H[i]), xv[st], b[i]);
      // step r -> r + 1: the first factors move up one output and the second ones
      // down one; the entries entering a lane come from its neighbours
      const float up = __shfl_up_sync(0xffffffffu, T[RB - 1], 1);
      const float dn = __shfl_down_sync(0xffffffffu, H[0], 1);
#pragma unroll
      for (int i = RB - 1; i > 0; --i) T[i] = T[i - 1];
#pragma unroll
      for (int i = 0; i + 1 < RB; ++i) H[i] = H[i + 1];
      T[0] = lane == 0 ? tl[st] : up;
      H[RB - 1] = lane == 31 ? hl[st] : dn;
    }
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const float y = __fsub_rn(b[i], cmp[i]);
      const float t = __fadd_rn(acc[i], y);
      cmp[i] = __fsub_rn(__fsub_rn(t, acc[i]), y);
      acc[i] = t;
    }
  }
  double* dst = part + (int64_t)blockIdx.y * part_n + ((int64_t)par * nch + tk.z) * H0;
#pragma unroll
  for (int i = 0; i < RB; ++i)
    if (o0 + i < Hp) dst[o0 + i] = (double)acc[i] - (double)cmp[i];
}

// out index q (k forward, n transposed), parity q & 1, position o = q >> 1: the
// chunk sums of its task column, in double.  A CTA takes 32 outputs; its 8 rows
// of threads sum the chunks c = c0 + row, c0 + row + 8, ... in ascending order,
// and the 8 row sums are added in row order, so the result is the same on every
// run and for any batch.
template <bool TRANS>
__global__ void __launch_bounds__(256) k_head_rb_reduce(const double* __restrict__ part, int64_t part_n, int rbc,
                                                        float* __restrict__ out, int64_t N, int64_t h, int scale_s,
                                                        double* __restrict__ hout, int64_t hs) {
  __shared__ double red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 32 + tx;
  double s = 0.0;
  if (q < h) {
    const int par = (int)(q & 1);
    const int64_t o = q >> 1;
    const int64_t Hp = (h - par + 1) / 2;
    const int64_t H0 = (h + 1) / 2;
    const int64_t nch = (H0 + rbc - 1) / rbc;
    const int64_t blk = o / RBW;
    // forward: chunks from the one holding the block's first output to the last;
    // transposed: chunks up to the one holding the block's last reduction index
    const int64_t c0 = TRANS ? 0 : (blk * RBW) / rbc;
    const int64_t c1 = TRANS ? (min(Hp, (blk + 1) * RBW) - 1) / rbc + 1 : (Hp + rbc - 1) / rbc;
    const double* src = part + (int64_t)blockIdx.y * part_n + (int64_t)par * nch * H0 + o;
    for (int64_t c = c0 + ty; c < c1; c += 8) s += src[c * H0];
  }
  red[ty][tx] = s;
  __syncthreads();
  if (ty != 0 || q >= h) return;
  double t = 0.0;
#pragma unroll
  for (int r = 0; r < 8; ++r) t += red[r][tx];
  if (!TRANS && q == 0) t *= 0.5;
  if (TRANS && scale_s) t *= (double)q + 0.5;
  if (hout)
    hout[(int64_t)blockIdx.y * hs + q] = t;
  else
    out[(int64_t)blockIdx.y * N + q] = (float)((double)out[(int64_t)blockIdx.y * N + q] + t);
}

}  // namespace

void head_rb_tasks(int64_t h, std::vector<int4>& fwd, std::vector<int4>& trn, int64_t* part_n, int* rbc_out) {
  // the longest chunk (fewest partial sums) that still gives every SM two CTAs of
  // 8 warp tasks in each direction, down to 32 reduction indices
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  const int64_t H0 = (h + 1) / 2;
  int rbc = 512;
  for (;; rbc /= 2) {
    fwd.clear();
    trn.clear();
    for (int par = 0; par < 2; ++par) {
      const int64_t Hp = (h - par + 1) / 2;
      const int64_t nblk = (Hp + RBW - 1) / RBW;
      const int64_t nchp = (Hp + rbc - 1) / rbc;
      for (int64_t b = 0; b < nblk; ++b) {
        for (int64_t c = (b * RBW) / rbc; c < nchp; ++c) fwd.push_back(make_int4(par, (int)b, (int)c, 0));
        const int64_t last = std::min(Hp, (b + 1) * RBW) - 1;
        for (int64_t c = 0; c <= last / rbc; ++c) trn.push_back(make_int4(par, (int)b, (int)c, 0));
      }
    }
    if (rbc <= 32 || (int64_t)fwd.size() >= 16 * (int64_t)sms) break;
  }
  const int64_t nch = (H0 + rbc - 1) / rbc;
  *part_n = 2 * nch * H0;
  *rbc_out = rbc;
}

int launch_head_tab_init(Plan& P) {
  const int64_t h = P.p.head;
  if (!P.head_tab || h == 0) return GBDLT_OK;
  k_head_tab_init<<<(unsigned)h, 256, 0, P.stream>>>(P.head_lam, P.head_off, P.head_tab, h);
  count_launch();
  if (P.head_tabT) {
    k_head_tabT_init<<<(unsigned)h, 256, 0, P.stream>>>(P.head_lam, P.head_offT, P.head_tabT, h);
    count_launch();
  }
  return check_launch();
}

// grid of k_head_mm: (output tiles x 2 parities, item tiles)
inline dim3 head_mm_grid(int64_t h, int64_t nb) {
  return dim3((unsigned)(2 * (((h + 1) / 2 + MMO - 1) / MMO)), (unsigned)((nb + MMB - 1) / MMB));
}

template <typename T>
int launch_head_fwd(Plan& P, const T* c, T* chat, int64_t nb, double* hout) {
  const int64_t h = P.p.head;
  if (h == 0) return GBDLT_OK;
  const T* lam = sizeof(T) == 8 ? (const T*)P.head_lam : (const T*)P.head_lamf;
  if (sizeof(T) == 4 && h <= kHeadMM) {
    k_head_mm<T, false><<<head_mm_grid(h, nb), 256, 0, P.stream>>>(c, chat, lam, P.p.N, h, 0, hout,
                                                                   P.p.N * (int64_t)sizeof(T) / 8, nb);
    launched(P, "head", (double)nb * 0.5 * (double)h * (double)h, (double)nb * (double)sizeof(T) * 2.0 * (double)h);
    return check_launch();
  }
  if constexpr (sizeof(T) == 4) {
    if (P.head_lamp) {
      k_head_rb<false><<<dim3((unsigned)((P.head_ntask_f + 7) / 8), (unsigned)nb), 256, 0, P.stream>>>(
          c, P.head_lamp, P.head_tasks, P.head_ntask_f, P.p.N, h, P.head_rbc, P.head_part, P.head_part_n);
      launched(P, "head", (double)nb * 0.5 * (double)h * (double)h, (double)nb * 4.0 * 2.0 * (double)h);
      k_head_rb_reduce<false><<<dim3((unsigned)((h + 31) / 32), (unsigned)nb), 256, 0, P.stream>>>(
          P.head_part, P.head_part_n, P.head_rbc, chat, P.p.N, h, 0, hout, P.p.N * (int64_t)sizeof(T) / 8);
      launched(P, "head_reduce", 0.0, (double)nb * 8.0 * (double)P.head_part_n);
      return check_launch();
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (P.head_tab && !hout) {
      k_head_fwd_tab<<<dim3((unsigned)((h + HW - 1) / HW), (unsigned)nb), HW * 32, 0, P.stream>>>(
          c, chat, P.head_tab, P.head_off, P.p.N, h);
      launched(P, "head", (double)nb * 0.5 * (double)h * (double)h, (double)nb * 8.0 * 0.25 * (double)h * (double)h);
      return check_launch();
    }
  }
  k_head_fwd<T><<<dim3((unsigned)((h + HW - 1) / HW), (unsigned)nb), HW * 32, 0, P.stream>>>(
      c, chat, lam, P.p.N, h, hout, P.p.N * (int64_t)sizeof(T) / 8);
  launched(P, "head", (double)nb * 0.5 * (double)h * (double)h,
           (double)nb * (double)sizeof(T) * 3.0 * (double)h);
  return check_launch();
}

template <typename T>
int launch_head_t(Plan& P, const T* y, T* out, int scale_s, int64_t nb, double* hout) {
  const int64_t h = P.p.head;
  if (h == 0) return GBDLT_OK;
  const T* lam = sizeof(T) == 8 ? (const T*)P.head_lam : (const T*)P.head_lamf;
  if (sizeof(T) == 4 && h <= kHeadMM) {
    k_head_mm<T, true><<<head_mm_grid(h, nb), 256, 0, P.stream>>>(y, out, lam, P.p.N, h, scale_s, hout,
                                                                  P.p.N * (int64_t)sizeof(T) / 8, nb);
    launched(P, "head_t", (double)nb * 0.5 * (double)h * (double)h,
             (double)nb * (double)sizeof(T) * 2.0 * (double)h);
    return check_launch();
  }
  if constexpr (sizeof(T) == 4) {
    if (P.head_lamp) {
      k_head_rb<true><<<dim3((unsigned)((P.head_ntask_t + 7) / 8), (unsigned)nb), 256, 0, P.stream>>>(
          y, P.head_lamp, P.head_tasks + P.head_ntask_f, P.head_ntask_t, P.p.N, h, P.head_rbc, P.head_part,
          P.head_part_n);
      launched(P, "head_t", (double)nb * 0.5 * (double)h * (double)h, (double)nb * 4.0 * 2.0 * (double)h);
      k_head_rb_reduce<true><<<dim3((unsigned)((h + 31) / 32), (unsigned)nb), 256, 0, P.stream>>>(
          P.head_part, P.head_part_n, P.head_rbc, out, P.p.N, h, scale_s, hout, P.p.N * (int64_t)sizeof(T) / 8);
      launched(P, "head_reduce", 0.0, (double)nb * 8.0 * (double)P.head_part_n);
      return check_launch();
    }
  }
  if constexpr (sizeof(T) == 8) {
    if (P.head_tabT) {
      k_head_t_tabT<<<dim3((unsigned)((h + HW - 1) / HW), (unsigned)nb), HW * 32, 0, P.stream>>>(
          y, out, P.head_tabT, P.head_offT, P.p.N, h, scale_s, hout, P.p.N);
      launched(P, "head_t", (double)nb * 0.5 * (double)h * (double)h, (double)nb * 8.0 * 0.25 * (double)h * (double)h);
      return check_launch();
    }
    if (P.head_tab) {
      k_head_t_tab<<<dim3((unsigned)(2 * ((h + 63) / 64)), (unsigned)nb), TW * 32, 0, P.stream>>>(
          y, out, P.head_tab, P.head_off, P.p.N, h, scale_s, hout, P.p.N);
      launched(P, "head_t", (double)nb * 0.5 * (double)h * (double)h, (double)nb * 8.0 * 0.25 * (double)h * (double)h);
      return check_launch();
    }
  }
  k_head_t<T><<<dim3((unsigned)((h + HW - 1) / HW), (unsigned)nb), HW * 32, 0, P.stream>>>(
      y, out, lam, P.p.N, h, scale_s, hout, P.p.N * (int64_t)sizeof(T) / 8);
  launched(P, "head_t", (double)nb * 0.5 * (double)h * (double)h,
           (double)nb * (double)sizeof(T) * 3.0 * (double)h);
  return check_launch();
}

template int launch_head_fwd<double>(Plan&, const double*, double*, int64_t, double*);
template int launch_head_fwd<float>(Plan&, const float*, float*, int64_t, double*);
template int launch_head_t<double>(Plan&, const double*, double*, int, int64_t, double*);
template int launch_head_t<float>(Plan&, const float*, float*, int, int64_t, double*);

}  // namespace gbdlt
