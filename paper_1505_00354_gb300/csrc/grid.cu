// Fast path for N that is not a power of two.
//
// The FFT engine works on power-of-two lengths.  For other N the plan runs the
// chain of a plan on the power-of-two grid G > N (Sec. 2-4 unchanged on that
// grid):
//  * coefficient-space vectors are zero-padded to G: leg2cheb of the padded
//    vector is the Chebyshev expansion of the same degree-(N-1) polynomial, and
//    the transposed operators restricted to the first N columns are the N-point
//    ones (M is upper triangular, so M_N is the leading N x N block of M_G);
//  * the rows are the N-point Gauss-Legendre rule, not the grid: row k takes its
//    Taylor expansion (Eq. (6)-(8)) about the grid point j(k) nearest theta_k,
//    theta'_j = (j + 1/2) pi / G, with offset t_k = G (theta_k - theta'_j),
//    |t_k| <= pi/2, so |n dtheta_k| <= (N-1) pi / (2G) over the columns n < N
//    and L follows from Corollary 2.4 with that bound (plan.cu, derive_params).
//
// t_k is formed from the rule's own offset tN_k = N (theta_k - (k + 1/2) pi/N),
// which the node kernels compute to full relative accuracy:
//   t_k = (G/N) tN_k + pi ((2k + 1) G - (2j + 1) N) / (2N),
// the integer in the second term exact, so t_k carries no cancellation error.
//
// An inner plan may carry several rules at once (one per batch item): the batch
// executor runs every transform whose length lies in (G/2, G] through one chain
// on the grid G, each item with its own rule.
//
// The transposed Taylor prologue sums, per grid point, the rows mapped to it.
// Rows lie at least 3.11/(N + 1/2) apart in theta (the first gap, between the
// two smallest Bessel zeros scaled, is the narrowest) and grid cells are pi/G <
// pi/N wide, so a cell holds at most two rows; grid_attach checks it.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "gbdlt_internal.cuh"

namespace gbdlt {

namespace {

constexpr int TPB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + TPB - 1) / TPB); }

// nearest grid point and offset of every row
__global__ void k_grid_map(const double* __restrict__ theta, const double* __restrict__ tN, int64_t N, int64_t G,
                           int32_t* __restrict__ jmap, double* __restrict__ tr) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double scale = (double)G / (double)N;
  const double tk = tN[k];
  auto offset = [&](int64_t j) {
    const int64_t m = (2 * k + 1) * G - (2 * j + 1) * N;
    return scale * tk + M_PI * (double)m / (2.0 * (double)N);
  };
  int64_t j = (int64_t)floor(theta[k] * (double)G / M_PI);
  j = j < 0 ? 0 : (j > G - 1 ? G - 1 : j);
  double t = offset(j);
  // theta_k within a rounding of a cell edge: the other side's point is nearer
  if (t > 0.5 * M_PI && j + 1 < G) {
    ++j;
    t = offset(j);
  } else if (t < -0.5 * M_PI && j > 0) {
    --j;
    t = offset(j);
  }
  jmap[k] = (int32_t)j;
  tr[k] = t;
}

// kf[j] = first row k with jmap[k] >= j, j = 0..G (jmap is non-decreasing)
__global__ void k_grid_first(const int32_t* __restrict__ jmap, int64_t N, int64_t G, int32_t* __restrict__ kf) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j > G) return;
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if ((int64_t)jmap[mid] < j)
      lo = mid + 1;
    else
      hi = mid;
  }
  kf[j] = (int32_t)lo;
}

// largest number of rows on one grid point, and whether jmap is non-decreasing
__global__ void k_grid_check(const int32_t* __restrict__ jmap, const int32_t* __restrict__ kf, int64_t N, int64_t G,
                             int* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < G) atomicMax(out, kf[i + 1] - kf[i]);
  if (i + 1 < N && jmap[i + 1] < jmap[i]) atomicMax(out, 1 << 20);
}

template <typename T>
__global__ void k_grid_pad(const T* __restrict__ in, T* __restrict__ out, int64_t N, int64_t G) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= G) return;
  const int64_t bt = blockIdx.y;
  out[bt * G + i] = i < N ? in[bt * N + i] : (T)0;
}

template <typename T>
__global__ void k_grid_cut(const T* __restrict__ in, T* __restrict__ out, int64_t N, int64_t G) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t bt = blockIdx.y;
  out[bt * N + i] = in[bt * G + i];
}

// out_j = sum over the rows k of grid point j of g_k (w_k g_k when use_w), 0
// where no row falls; g and out have the grid's batch stride G
template <typename T>
__global__ void k_grid_scatter(const T* __restrict__ g, int use_w, const GridRule* __restrict__ rules,
                               const int32_t* __restrict__ item, T* __restrict__ out, int64_t G) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= G) return;
  const int64_t bt = blockIdx.y;
  const GridRule R = rules[item ? item[bt] : 0];
  g += bt * G;
  T s = (T)0;
  for (int64_t k = R.kf[j]; k < R.kf[j + 1]; ++k) s += use_w ? (T)((double)g[k] * R.w[k]) : g[k];
  out[bt * G + j] = s;
}

}  // namespace

struct GridRules {
  int64_t G = 0;
  std::vector<int64_t> n;
  void* block = nullptr;       // maps of every rule
  GridRule* dev = nullptr;     // [rules] (inside block)
  size_t bytes = 0;
};

double grid_bound(int64_t N, int64_t G) {
  return N == G ? 0.83845 : (double)(N - 1) * M_PI / (2.0 * (double)G) * (1.0 + 1e-9);
}

int grid_rules_create(int64_t G, const std::vector<Plan*>& nodes, cudaStream_t s, GridRules** out) {
  *out = nullptr;
  if (nodes.empty() || G < 2 || (G & (G - 1))) return GBDLT_ERR_INVALID_ARG;
  GridRules* R = new (std::nothrow) GridRules();
  if (!R) return GBDLT_ERR_OOM;
  R->G = G;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t nr = nodes.size();
  std::vector<size_t> oj(nr), ot(nr), okf(nr);
  size_t off = al(sizeof(GridRule) * nr) + al(sizeof(int));
  for (size_t r = 0; r < nr; ++r) {
    const int64_t N = nodes[r]->p.N;
    if (N < 1 || N > G) {
      delete R;
      return GBDLT_ERR_INVALID_ARG;
    }
    R->n.push_back(N);
    oj[r] = off;
    off += al(sizeof(int32_t) * N);
    ot[r] = off;
    off += al(sizeof(double) * N);
    okf[r] = off;
    off += al(sizeof(int32_t) * (G + 1));
  }
  R->bytes = off;
  if (dev_malloc(&R->block, off) != cudaSuccess) {
    cudaGetLastError();
    delete R;
    return GBDLT_ERR_OOM;
  }
  char* base = (char*)R->block;
  R->dev = (GridRule*)base;
  int* chk = (int*)(base + al(sizeof(GridRule) * nr));
  std::vector<GridRule> host(nr);
  bool ok = cudaMemsetAsync(chk, 0, sizeof(int), s) == cudaSuccess;
  for (size_t r = 0; r < nr && ok; ++r) {
    const Plan& P = *nodes[r];
    const int64_t N = P.p.N;
    int32_t* jm = (int32_t*)(base + oj[r]);
    double* tr = (double*)(base + ot[r]);
    int32_t* kf = (int32_t*)(base + okf[r]);
    host[r] = GridRule{N, jm, tr, kf, P.w};
    k_grid_map<<<nblk(N), TPB, 0, s>>>(P.theta, P.tN, N, G, jm, tr);
    k_grid_first<<<nblk(G + 1), TPB, 0, s>>>(jm, N, G, kf);
    k_grid_check<<<nblk(std::max(G, N)), TPB, 0, s>>>(jm, kf, N, G, chk);
    count_launch(3);
    ok = check_launch() == GBDLT_OK;
  }
  int worst = 0;
  if (!ok || cudaMemcpyAsync(R->dev, host.data(), sizeof(GridRule) * nr, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpy(&worst, chk, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    grid_rules_free(R);
    return GBDLT_ERR_CUDA;
  }
  // more than two rows on a grid point (or rows out of order) would break the
  // transposed prologue's two slots per point
  if (worst > 2) {
    grid_rules_free(R);
    return GBDLT_ERR_UNIMPLEMENTED;
  }
  *out = R;
  return GBDLT_OK;
}

void grid_rules_free(GridRules* r) {
  if (!r) return;
  if (r->block) cudaFree(r->block);
  delete r;
}

size_t grid_rules_bytes(const GridRules* r) { return r ? r->bytes : 0; }

int grid_attach(Plan& I, GridRules* R, const int32_t* item, bool own) {
  if (!R || R->G != I.p.N) return GBDLT_ERR_INVALID_ARG;
  const size_t ts = I.p.prec == GBDLT_FP64 ? sizeof(double) : sizeof(float);
  if (!I.rg_g && dev_malloc(&I.rg_g, ts * (size_t)I.bcap * (size_t)I.p.N) != cudaSuccess) {
    cudaGetLastError();
    return GBDLT_ERR_OOM;
  }
  I.rg_rules = R->dev;
  I.rg_item = item;
  I.rg_item0 = 0;
  I.rg_nmax = 0;
  for (int64_t n : R->n) I.rg_nmax = std::max(I.rg_nmax, n);
  if (own) I.rg_own = R;
  return GBDLT_OK;
}

template <typename T>
int launch_grid_pad(Plan& P, const T* in, T* out, int64_t N, int64_t G, int64_t nb) {
  k_grid_pad<T><<<dim3(nblk(G), (unsigned)nb), TPB, 0, P.stream>>>(in, out, N, G);
  launched(P, "grid_pad", 0.0, (double)nb * (double)sizeof(T) * (double)(N + G));
  return check_launch();
}

template <typename T>
int launch_grid_cut(Plan& P, const T* in, T* out, int64_t N, int64_t G, int64_t nb) {
  k_grid_cut<T><<<dim3(nblk(N), (unsigned)nb), TPB, 0, P.stream>>>(in, out, N, G);
  launched(P, "grid_cut", 0.0, (double)nb * (double)sizeof(T) * 2.0 * (double)N);
  return check_launch();
}

template <typename T>
int launch_grid_scatter(Plan& I, const T* g, int use_w, T* out, int64_t nb) {
  const int64_t G = I.p.N;
  k_grid_scatter<T><<<dim3(nblk(G), (unsigned)nb), TPB, 0, I.stream>>>(
      g, use_w, I.rg_rules, I.rg_item ? I.rg_item + I.rg_item0 : nullptr, out, G);
  launched(I, "grid_scatter", (double)nb * (double)I.rg_nmax, (double)nb * (double)sizeof(T) * (double)(I.rg_nmax + G));
  return check_launch();
}

template int launch_grid_pad<double>(Plan&, const double*, double*, int64_t, int64_t, int64_t);
template int launch_grid_pad<float>(Plan&, const float*, float*, int64_t, int64_t, int64_t);
template int launch_grid_cut<double>(Plan&, const double*, double*, int64_t, int64_t, int64_t);
template int launch_grid_cut<float>(Plan&, const float*, float*, int64_t, int64_t, int64_t);
template int launch_grid_scatter<double>(Plan&, const double*, int, double*, int64_t);
template int launch_grid_scatter<float>(Plan&, const float*, int, float*, int64_t);

}  // namespace gbdlt
