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
// twiddle from a two-level table of e^{2 pi i e/N}.
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

// multiply by e^{DIR i a} given (cos a, sin a)
template <typename T, int DIR>
__device__ __forceinline__ C2<T> rot(C2<T> v, T c, T s) {
  const T sd = DIR > 0 ? s : -s;
  return mk<T>(v.x * c - v.y * sd, v.x * sd + v.y * c);
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

// One Stockham stage of radix R over `lines` vectors of length L (current
// sub-transform length Ns): butterfly j reads x[j + r L/R], applies
// w_{Ns R}^{r (j mod Ns)}, takes the R-point DFT and writes
// y[(j / Ns) Ns R + (j mod Ns) + r Ns].  Twiddles come from the 4096-entry
// table; in FP32 only the power-of-two multiples are loaded and the rest are
// products of them (FP32 arithmetic is cheap, table traffic is not).
template <typename T, int DIR, int R>
__device__ __forceinline__ void stage(C2<T>* sm, int L, int logL, int lines, int LP, int Ns,
                                      const C2<T>* __restrict__ tw) {
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
          if (sizeof(T) == 8 || (r & (r - 1)) == 0) {
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

// In-place FFT of `lines` vectors of length L held at sidx(line, LP, i):
// one stage of radix 2^(log2 L mod 4) (if any), then radix-16 stages.
template <typename T, int DIR>
__device__ void fft_tile(C2<T>* sm, int L, int logL, int lines, int LP, const C2<T>* __restrict__ tw) {
  int Ns = 1;
  const int rem = logL & 3;
  if (rem == 1) {
    stage<T, DIR, 2>(sm, L, logL, lines, LP, Ns, tw);
    Ns = 2;
  } else if (rem == 2) {
    stage<T, DIR, 4>(sm, L, logL, lines, LP, Ns, tw);
    Ns = 4;
  } else if (rem == 3) {
    stage<T, DIR, 8>(sm, L, logL, lines, LP, Ns, tw);
    Ns = 8;
  }
  while (Ns < L) {
    stage<T, DIR, 16>(sm, L, logL, lines, LP, Ns, tw);
    Ns <<= 4;
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_single(C2<T>* __restrict__ data, int L, int logL, int64_t nvec, const C2<T>* __restrict__ tw4096) {
  extern __shared__ unsigned char smraw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int lines_max = FFT_TILE / L;
  const int64_t v0 = (int64_t)blockIdx.x * lines_max;
  const int lines = (int)min((int64_t)lines_max, nvec - v0);
  const int LP = line_pitch(L);
  const int tot = lines * L;
  C2<T>* g = data + v0 * L;
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) sm[sidx(i >> logL, LP, i & (L - 1))] = g[i];
  __syncthreads();
  fft_tile<T, DIR>(sm, L, logL, lines, LP, tw4096);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) g[i] = sm[sidx(i >> logL, LP, i & (L - 1))];
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_cols(C2<T>* __restrict__ data, int64_t N, int L1, int logL1, int L2, int C, int logC,
               const C2<T>* __restrict__ tw4096, const C2<T>* __restrict__ thi,
               const C2<T>* __restrict__ tlo) {
  extern __shared__ unsigned char smraw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int c0 = blockIdx.x * C;
  C2<T>* g = data + (int64_t)blockIdx.y * N;
  const int LP = line_pitch(L1);
  const int tot = L1 * C;
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    const int n1 = i >> logC, c = i & (C - 1);
    sm[sidx(c, LP, n1)] = g[(int64_t)n1 * L2 + c0 + c];
  }
  __syncthreads();
  fft_tile<T, DIR>(sm, L1, logL1, C, LP, tw4096);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    const int k1 = i >> logC, c = i & (C - 1);
    const int64_t e = (int64_t)(c0 + c) * k1;
    C2<T> val = sm[sidx(c, LP, k1)];
    if (e != 0) {
      const C2<T> w = tw_lookup<T>(thi, tlo, e);
      val = cmul<T>(val, mk<T>(w.x, DIR > 0 ? w.y : -w.y));
    }
    g[(int64_t)k1 * L2 + c0 + c] = val;
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_rows(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, int64_t N, int L1, int L2,
               int logL2, int C2n, int logC2, const C2<T>* __restrict__ tw4096) {
  extern __shared__ unsigned char smraw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int r0 = blockIdx.x * C2n;
  const C2<T>* g = in + (int64_t)blockIdx.y * N;
  C2<T>* o = out + (int64_t)blockIdx.y * N;
  const int LP = line_pitch(L2);
  const int tot = L2 * C2n;
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    const int line = i >> logL2, n2 = i & (L2 - 1);
    sm[sidx(line, LP, n2)] = g[(int64_t)(r0 + line) * L2 + n2];
  }
  __syncthreads();
  fft_tile<T, DIR>(sm, L2, logL2, C2n, LP, tw4096);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    const int k2 = i >> logC2, line = i & (C2n - 1);
    o[(int64_t)(r0 + line) + (int64_t)L1 * k2] = sm[sidx(line, LP, k2)];
  }
}

template <typename T, int DIR>
static void* fft_dir(Plan& P, void* a, void* b, int64_t nvec) {
  using CT = C2<T>;
  const int64_t N = P.p.N;
  if (nvec <= 0 || N <= 1) return a;
  const TwT<T> tw = tw_tables(P, T());
  const size_t smax = (size_t)FFT_SMEM_ELEMS * sizeof(CT);
  static bool attrs = false;  // one flag per (T, DIR) instantiation
  if (!attrs) {
    cudaFuncSetAttribute(k_fft_single<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    cudaFuncSetAttribute(k_fft_cols<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    cudaFuncSetAttribute(k_fft_rows<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    attrs = true;
  }
  if (N <= FFT_TILE) {
    int L = (int)N;
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    int lines = FFT_TILE / L;
    int64_t grid = (nvec + lines - 1) / lines;
    size_t sm = (size_t)lines * line_pitch(L) * sizeof(CT);
    k_fft_single<T, DIR><<<(unsigned)grid, FFT_THREADS, sm, P.stream>>>((CT*)a, L, lg, nvec, tw.t4096);
    launched(P, "fft_single", 5.0 * (double)N * lg * nvec, 2.0 * (double)nvec * N * sizeof(CT));
    return a;
  }
  int p = 0;
  while ((1ll << p) < N) ++p;
  int L1 = 1 << (p / 2);
  int L2 = (int)(N / L1);
  int C = FFT_TILE / L1;
  int C2n = FFT_TILE / L2;
  int lL1 = p / 2, lL2 = p - p / 2, lC = 12 - lL1, lC2 = 12 - lL2;
  dim3 g1(L2 / C, (unsigned)nvec);
  k_fft_cols<T, DIR><<<g1, FFT_THREADS, (size_t)C * line_pitch(L1) * sizeof(CT), P.stream>>>(
      (CT*)a, N, L1, lL1, L2, C, lC, tw.t4096, tw.nhi, tw.nlo);
  launched(P, "fft_cols", (5.0 * (p / 2) + 6.0) * (double)N * nvec, 2.0 * (double)nvec * N * sizeof(CT));
  dim3 g2(L1 / C2n, (unsigned)nvec);
  k_fft_rows<T, DIR><<<g2, FFT_THREADS, (size_t)C2n * line_pitch(L2) * sizeof(CT), P.stream>>>(
      (const CT*)a, (CT*)b, N, L1, L2, lL2, C2n, lC2, tw.t4096);
  launched(P, "fft_rows", 5.0 * (p - p / 2) * (double)N * nvec, 2.0 * (double)nvec * N * sizeof(CT));
  return b;
}

template <typename T>
void* launch_fft(Plan& P, void* a, void* b, int64_t nvec, int dir) {
  return dir > 0 ? fft_dir<T, 1>(P, a, b, nvec) : fft_dir<T, -1>(P, a, b, nvec);
}

template void* launch_fft<double>(Plan&, void*, void*, int64_t, int);
template void* launch_fft<float>(Plan&, void*, void*, int64_t, int);

}  // namespace gbdlt
