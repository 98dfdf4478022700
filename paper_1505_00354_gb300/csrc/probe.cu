// FP64 arithmetic-rate probe: the denominator of the roofline of the FP64
// kernels (their bound is the FP64 pipe, whose rate no driver-side measurement
// covers).  Every thread runs 8 independent chains of fused multiply-adds whose
// values stay finite (a contraction towards a fixed point), over a grid of 8
// CTAs of 256 threads per SM; the rate is 2 flops per FMA over the kernel's
// duration by CUDA events.  The loop count is fixed: the kernel always ends.
#include "gbdlt_internal.cuh"

namespace gbdlt {

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_probe(double* __restrict__ out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // one store per CTA keeps the chains live without a write per thread
  if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

}  // namespace gbdlt

using namespace gbdlt;

extern "C" int gbdlt_fp64_fma_rate(void* cuda_stream, double* flops_per_second) {
  if (!flops_per_second) return GBDLT_ERR_INVALID_ARG;
  *flops_per_second = 0.0;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    return GBDLT_ERR_CUDA;
  }
  double* out = nullptr;
  if (dev_malloc((void**)&out, sizeof(double) * 8 * (size_t)sms) != cudaSuccess) {
    cudaGetLastError();
    return GBDLT_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = GBDLT_OK;
  const unsigned grid = 8u * (unsigned)sms;
  const int iters = 4096;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = GBDLT_ERR_CUDA;
  float best = 0.f;
  for (int rep = 0; rep < 4 && st == GBDLT_OK; ++rep) {
    cudaEventRecord(e0, s);
    k_fma_probe<<<grid, 256, 0, s>>>(out, iters, 0.999999, 1e-6);
    cudaEventRecord(e1, s);
    count_launch();
    float ms = 0.f;
    if (check_launch() || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = GBDLT_ERR_CUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // the first run warms up
  }
  if (st == GBDLT_OK && best > 0.f)
    *flops_per_second = 2.0 * (double)kChains * iters * 256.0 * grid / (best * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  cudaGetLastError();
  return st;
}
