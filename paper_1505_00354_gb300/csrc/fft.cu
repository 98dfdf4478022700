// Batched complex FFT of power-of-two length N on one GPU.
//
// This is the transform engine behind every DCT/DST of the method (Sec. 2.3,
// Eq. 13; the DCT/DST are reduced to complex FFTs of length N by the pre- and
// post-processing kernels in stages.cu).  Sign convention: DIR = +1 computes
// y_k = sum_n x_n e^{+2 pi i nk/N}, DIR = -1 the conjugate kernel; no scaling.
//
// Layout: nvec vectors, each N contiguous complex values (float2/double2).
//  * N <= 4096: one pass; a CTA holds 4096/N vectors in shared memory and runs
//    an in-place Stockham autosort FFT (radix-4 stages, one radix-2 stage when
//    log2 N is odd).
//  * N > 4096: four-step with N = L1 * L2 (L1, L2 <= 4096).  Pass 1 ("columns"):
//    a CTA loads C = 4096/L1 adjacent columns n2 (C contiguous elements per
//    row, so global loads and stores are coalesced segments), transforms along
//    n1, multiplies by e^{DIR 2 pi i n2 k1 / N} and stores in place.  Pass 2
//    ("rows"): a CTA loads C2 = 4096/L2 contiguous rows k1, transforms along
//    n2 and stores X[k1 + L1 k2] into the second buffer, C2 contiguous elements
//    per k2.
// Twiddles come from tables (no FP64 trigonometry in the hot loop): the inner
// Stockham twiddles from a 4096-entry table e^{2 pi i j/4096}, the inter-pass
// twiddle from a two-level table of e^{2 pi i e/N}.
#include "gbdlt_internal.cuh"

namespace gbdlt {

constexpr int FFT_TILE = 4096;
constexpr int FFT_THREADS = 256;

// e^{2 pi i e / N} from the two-level table, multiplied in the precision T
template <typename T>
__device__ __forceinline__ C2<T> tw_lookup(const C2<T>* __restrict__ hi, const C2<T>* __restrict__ lo,
                                           int64_t e) {
  return cmul<T>(hi[e >> 12], lo[e & 4095]);
}

// In-place Stockham FFT of `lines` vectors of length L stored at
// sm[line * pitch + i].  All threads of the CTA must call it.
template <typename T, int DIR>
__device__ void fft_tile(C2<T>* sm, int L, int lines, int pitch,
                         const C2<T>* __restrict__ tw4096) {
  using CT = C2<T>;
  const int tid = threadIdx.x;
  int logL = 31 - __clz(L);
  int Ns = 1;
  int rem = logL;
  while (Ns < L) {
    if (rem >= 2) {
      constexpr int PER = FFT_TILE / 4 / FFT_THREADS;  // butterflies per thread
      const int Lq = L >> 2;
      const int nbf = lines * Lq;
      CT v[PER][4];
      int dst[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        int b = tid + q * FFT_THREADS;
        dst[q] = -1;
        if (b < nbf) {
          int line = b / Lq;
          int j = b - line * Lq;
          int k = j & (Ns - 1);
          CT* base = sm + line * pitch;
#pragma unroll
          for (int r = 0; r < 4; ++r) v[q][r] = base[j + r * Lq];
          if (Ns > 1) {
            int step = (FFT_TILE / 4) / Ns;  // 4096 / (Ns * 4)
#pragma unroll
            for (int r = 1; r < 4; ++r) {
              const CT w = tw4096[r * k * step];
              const CT wt = mk<T>(w.x, DIR > 0 ? w.y : -w.y);
              v[q][r] = cmul<T>(v[q][r], wt);
            }
          }
          dst[q] = line * pitch + (j - k) * 4 + k;  // (j/Ns)*Ns*4 + k
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        if (dst[q] >= 0) {
          CT a0 = v[q][0], a1 = v[q][1], a2 = v[q][2], a3 = v[q][3];
          CT s02 = cadd<T>(a0, a2), d02 = csub<T>(a0, a2);
          CT s13 = cadd<T>(a1, a3), d13 = cmul_i<T, DIR>(csub<T>(a1, a3));
          CT* o = sm + dst[q];
          o[0] = cadd<T>(s02, s13);
          o[Ns] = cadd<T>(d02, d13);
          o[2 * Ns] = csub<T>(s02, s13);
          o[3 * Ns] = csub<T>(d02, d13);
        }
      }
      __syncthreads();
      Ns <<= 2;
      rem -= 2;
    } else {
      constexpr int PER = FFT_TILE / 2 / FFT_THREADS;
      const int Lh = L >> 1;
      const int nbf = lines * Lh;
      CT v[PER][2];
      int dst[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        int b = tid + q * FFT_THREADS;
        dst[q] = -1;
        if (b < nbf) {
          int line = b / Lh;
          int j = b - line * Lh;
          int k = j & (Ns - 1);
          CT* base = sm + line * pitch;
          v[q][0] = base[j];
          v[q][1] = base[j + Lh];
          if (Ns > 1) {
            const CT w = tw4096[k * ((FFT_TILE / 2) / Ns)];
            const CT wt = mk<T>(w.x, DIR > 0 ? w.y : -w.y);
            v[q][1] = cmul<T>(v[q][1], wt);
          }
          dst[q] = line * pitch + (j - k) * 2 + k;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        if (dst[q] >= 0) {
          CT* o = sm + dst[q];
          CT a0 = v[q][0], a1 = v[q][1];
          o[0] = cadd<T>(a0, a1);
          o[Ns] = csub<T>(a0, a1);
        }
      }
      __syncthreads();
      Ns <<= 1;
      rem -= 1;
    }
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_single(C2<T>* __restrict__ data, int L, int64_t nvec, const C2<T>* __restrict__ tw4096) {
  extern __shared__ unsigned char smraw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int lines_max = FFT_TILE / L;
  const int64_t v0 = (int64_t)blockIdx.x * lines_max;
  const int lines = (int)min((int64_t)lines_max, nvec - v0);
  const int pitch = L;
  const int tot = lines * L;
  C2<T>* g = data + v0 * L;
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) sm[i] = g[i];
  __syncthreads();
  fft_tile<T, DIR>(sm, L, lines, pitch, tw4096);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) g[i] = sm[i];
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_cols(C2<T>* __restrict__ data, int64_t N, int L1, int L2, int C,
               const C2<T>* __restrict__ tw4096, const C2<T>* __restrict__ thi,
               const C2<T>* __restrict__ tlo) {
  extern __shared__ unsigned char smraw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int c0 = blockIdx.x * C;
  C2<T>* g = data + (int64_t)blockIdx.y * N;
  const int pitch = L1 + 1;
  const int tot = L1 * C;
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    int n1 = i / C, c = i - n1 * C;
    sm[c * pitch + n1] = g[(int64_t)n1 * L2 + c0 + c];
  }
  __syncthreads();
  fft_tile<T, DIR>(sm, L1, C, pitch, tw4096);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    int k1 = i / C, c = i - k1 * C;
    int64_t e = (int64_t)(c0 + c) * k1;
    C2<T> val = sm[c * pitch + k1];
    if (e != 0) {
      const C2<T> w = tw_lookup<T>(thi, tlo, e);
      const C2<T> wt = mk<T>(w.x, DIR > 0 ? w.y : -w.y);
      val = cmul<T>(val, wt);
    }
    g[(int64_t)k1 * L2 + c0 + c] = val;
  }
}

template <typename T, int DIR>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_rows(const C2<T>* __restrict__ in, C2<T>* __restrict__ out, int64_t N, int L1, int L2,
               int C2n, const C2<T>* __restrict__ tw4096) {
  extern __shared__ unsigned char smraw[];
  C2<T>* sm = reinterpret_cast<C2<T>*>(smraw);
  const int r0 = blockIdx.x * C2n;
  const C2<T>* g = in + (int64_t)blockIdx.y * N;
  C2<T>* o = out + (int64_t)blockIdx.y * N;
  const int pitch = L2 + 1;
  const int tot = L2 * C2n;
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    int line = i / L2, n2 = i - line * L2;
    sm[line * pitch + n2] = g[(int64_t)(r0 + line) * L2 + n2];
  }
  __syncthreads();
  fft_tile<T, DIR>(sm, L2, C2n, pitch, tw4096);
  for (int i = threadIdx.x; i < tot; i += FFT_THREADS) {
    int k2 = i / C2n, line = i - k2 * C2n;
    o[(int64_t)(r0 + line) + (int64_t)L1 * k2] = sm[line * pitch + k2];
  }
}

template <typename T, int DIR>
static void* fft_dir(Plan& P, void* a, void* b, int64_t nvec) {
  using CT = C2<T>;
  const int64_t N = P.p.N;
  if (nvec <= 0 || N <= 1) return a;
  const TwT<T> tw = tw_tables(P, T());
  // largest tile: C lines of L1+1 (pitch) with C * L1 = 4096 and L1 >= 64
  const size_t smax = (size_t)(FFT_TILE + 64) * sizeof(CT);
  static bool attrs = false;  // one flag per (T, DIR) instantiation
  if (!attrs) {
    cudaFuncSetAttribute(k_fft_single<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    cudaFuncSetAttribute(k_fft_cols<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    cudaFuncSetAttribute(k_fft_rows<T, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    attrs = true;
  }
  if (N <= FFT_TILE) {
    int L = (int)N;
    int lines = FFT_TILE / L;
    int64_t grid = (nvec + lines - 1) / lines;
    size_t sm = (size_t)lines * L * sizeof(CT);
    k_fft_single<T, DIR><<<(unsigned)grid, FFT_THREADS, sm, P.stream>>>((CT*)a, L, nvec, tw.t4096);
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    launched(P, "fft_single", 5.0 * (double)N * lg * nvec, 2.0 * (double)nvec * N * sizeof(CT));
    return a;
  }
  int p = 0;
  while ((1ll << p) < N) ++p;
  int L1 = 1 << (p / 2);
  int L2 = (int)(N / L1);
  int C = FFT_TILE / L1;
  int C2n = FFT_TILE / L2;
  dim3 g1(L2 / C, (unsigned)nvec);
  k_fft_cols<T, DIR><<<g1, FFT_THREADS, (size_t)C * (L1 + 1) * sizeof(CT), P.stream>>>(
      (CT*)a, N, L1, L2, C, tw.t4096, tw.nhi, tw.nlo);
  launched(P, "fft_cols", (5.0 * (p / 2) + 6.0) * (double)N * nvec, 2.0 * (double)nvec * N * sizeof(CT));
  dim3 g2(L1 / C2n, (unsigned)nvec);
  k_fft_rows<T, DIR><<<g2, FFT_THREADS, (size_t)C2n * (L2 + 1) * sizeof(CT), P.stream>>>(
      (const CT*)a, (CT*)b, N, L1, L2, C2n, tw.t4096);
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
