// Uneven batches: many transforms of different lengths and directions run as
// one CUDA-graph replay.
//
// The transforms are grouped by (N, direction).  Each distinct N gets one plan
// whose workspace holds the largest group of that N in one pass, so a group is
// a single batched chain (every stage kernel carries the batch index in
// blockIdx.y and every FFT launch transforms all vectors of the group).  At
// creation the group chains are run once (to settle kernel attributes) and then
// captured from an internal stream into one CUDA graph.  An execution is: wait
// for the caller's stream, gather the caller's concatenated inputs into the
// grouped staging layout, replay the graph, scatter the grouped outputs back to
// the caller's layout, and make the caller's stream wait for the result.
// Nothing is allocated per execution.
#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "gbdlt_internal.cuh"

namespace gbdlt {

struct BatchGroup {
  int64_t N;
  int dir;  // 0: DLT, 1: IDLT
  int64_t count;
  int64_t stage_off;  // element offset of the group's first vector in the staging buffers
  Plan* plan;
};

struct Batch {
  int prec = GBDLT_FP64;
  int64_t B = 0, total = 0, maxN = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<Plan*> plans;
  std::vector<BatchGroup> groups;
  int64_t* d_src = nullptr;    // [B] offset of transform i in the caller's layout
  int64_t* d_stage = nullptr;  // [B] offset of transform i in the staging layout
  int64_t* d_len = nullptr;    // [B] N_i
  void* stage_in = nullptr;
  void* stage_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;  // kernel nodes one replay launches
};

namespace {

template <typename E>
__global__ void k_batch_move(const E* __restrict__ src, E* __restrict__ dst, const int64_t* __restrict__ src_off,
                             const int64_t* __restrict__ dst_off, const int64_t* __restrict__ len) {
  const int64_t i = blockIdx.y;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < len[i]) dst[dst_off[i] + j] = src[src_off[i] + j];
}

int move(Batch& b, const void* src, void* dst, bool gather) {
  const int64_t* so = gather ? b.d_src : b.d_stage;
  const int64_t* dso = gather ? b.d_stage : b.d_src;
  dim3 grid((unsigned)((b.maxN + 255) / 256), (unsigned)b.B);
  if (b.prec == GBDLT_FP64)
    k_batch_move<double><<<grid, 256, 0, b.s>>>((const double*)src, (double*)dst, so, dso, b.d_len);
  else
    k_batch_move<float><<<grid, 256, 0, b.s>>>((const float*)src, (float*)dst, so, dso, b.d_len);
  count_launch();
  return check_launch();
}

int run_groups(Batch& b) {
  const size_t es = b.prec == GBDLT_FP64 ? 8 : 4;
  for (const BatchGroup& g : b.groups) {
    const char* in = (const char*)b.stage_in + (size_t)g.stage_off * es;
    char* out = (char*)b.stage_out + (size_t)g.stage_off * es;
    int st = run_op(reinterpret_cast<gbdlt_plan>(g.plan), g.dir ? OP_IDLT : OP_DLT, in, out, g.count);
    if (st) return st;
  }
  return GBDLT_OK;
}

void free_batch(Batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (Plan* p : b->plans) free_plan(p);
  if (b->d_src) cudaFree(b->d_src);
  if (b->stage_in) cudaFree(b->stage_in);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->s) cudaStreamDestroy(b->s);
  delete b;
}

}  // namespace

}  // namespace gbdlt

using namespace gbdlt;

struct gbdlt_batch_s {};  // opaque tag; the pointer is a gbdlt::Batch

extern "C" int gbdlt_batch_create(const int64_t* Ns_host, const int32_t* dirs_host, int64_t B, int prec,
                                  double eps, gbdlt_batch* out) {
  if (!out) return GBDLT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!Ns_host || !dirs_host || B < 1 || B > 65535) return GBDLT_ERR_INVALID_ARG;
  if (prec != GBDLT_FP64 && prec != GBDLT_FP32) return GBDLT_ERR_INVALID_ARG;
  for (int64_t i = 0; i < B; ++i) {
    const int64_t N = Ns_host[i];
    if (N < 1 || N > (1ll << 24) || (N & (N - 1))) return GBDLT_ERR_UNSUPPORTED_N;
    if (dirs_host[i] != 0 && dirs_host[i] != 1) return GBDLT_ERR_INVALID_ARG;
  }
  Batch* b = new (std::nothrow) Batch();
  if (!b) return GBDLT_ERR_OOM;
  b->prec = prec;
  b->B = B;
  const size_t es = prec == GBDLT_FP64 ? 8 : 4;
  auto fail = [&](int st) {
    cudaGetLastError();
    free_batch(b);
    return st;
  };
  if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail(GBDLT_ERR_CUDA);
  // groups by (N, dir), staging offsets, per-transform offsets
  std::map<std::pair<int64_t, int>, std::vector<int64_t>> members;
  std::vector<int64_t> src(B), stage(B), len(B);
  int64_t off = 0;
  for (int64_t i = 0; i < B; ++i) {
    src[i] = off;
    len[i] = Ns_host[i];
    off += Ns_host[i];
    b->maxN = std::max(b->maxN, Ns_host[i]);
    members[{Ns_host[i], dirs_host[i]}].push_back(i);
  }
  b->total = off;
  std::map<int64_t, int64_t> max_count;
  for (auto& kv : members)
    max_count[kv.first.first] = std::max<int64_t>(max_count[kv.first.first], (int64_t)kv.second.size());
  std::map<int64_t, Plan*> plan_of;
  for (auto& kv : max_count) {
    Plan* p = nullptr;
    int st = plan_create_impl(kv.first, prec, eps, b->s, kv.second, &p);
    if (st) return fail(st);
    b->plans.push_back(p);
    plan_of[kv.first] = p;
  }
  int64_t soff = 0;
  for (auto& kv : members) {
    BatchGroup g;
    g.N = kv.first.first;
    g.dir = kv.first.second;
    g.count = (int64_t)kv.second.size();
    g.stage_off = soff;
    g.plan = plan_of[g.N];
    for (size_t q = 0; q < kv.second.size(); ++q) stage[kv.second[q]] = soff + (int64_t)q * g.N;
    soff += g.count * g.N;
    b->groups.push_back(g);
  }
  // device tables and staging
  if (cudaMalloc(&b->d_src, sizeof(int64_t) * 3 * (size_t)B) != cudaSuccess) return fail(GBDLT_ERR_OOM);
  b->d_stage = b->d_src + B;
  b->d_len = b->d_src + 2 * B;
  if (cudaMalloc(&b->stage_in, 2 * es * (size_t)b->total) != cudaSuccess) return fail(GBDLT_ERR_OOM);
  b->stage_out = (char*)b->stage_in + es * (size_t)b->total;
  if (cudaMemcpy(b->d_src, src.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_stage, stage.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_len, len.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemsetAsync(b->stage_in, 0, 2 * es * (size_t)b->total, b->s) != cudaSuccess)
    return fail(GBDLT_ERR_CUDA);
  // one plain run (kernel attributes, lazy module loading), then capture
  int st = run_groups(*b);
  if (st) return fail(st);
  if (cudaStreamSynchronize(b->s) != cudaSuccess) return fail(GBDLT_ERR_CUDA);
  if (cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(GBDLT_ERR_CUDA);
  st = run_groups(*b);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->s, &graph);
  if (st || ce != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    return fail(st ? st : GBDLT_ERR_CUDA);
  }
  b->graph = graph;
  if (cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) return fail(GBDLT_ERR_CUDA);
  {
    size_t n = 0;
    if (cudaGraphGetNodes(graph, nullptr, &n) != cudaSuccess) return fail(GBDLT_ERR_CUDA);
    std::vector<cudaGraphNode_t> nodes(n);
    if (n && cudaGraphGetNodes(graph, nodes.data(), &n) != cudaSuccess) return fail(GBDLT_ERR_CUDA);
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->graph_kernels;
    }
  }
  *out = reinterpret_cast<gbdlt_batch>(b);
  return GBDLT_OK;
}

extern "C" int gbdlt_batch_exec(gbdlt_batch batch, const void* in, void* out, void* cuda_stream) {
  if (!batch || !in || !out) return GBDLT_ERR_INVALID_ARG;
  Batch& b = *reinterpret_cast<Batch*>(batch);
  cudaStream_t user = (cudaStream_t)cuda_stream;
  if (cudaEventRecord(b.ev_in, user) != cudaSuccess || cudaStreamWaitEvent(b.s, b.ev_in, 0) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  int st = move(b, in, b.stage_in, true);
  if (st) return st;
  if (cudaGraphLaunch(b.exec, b.s) != cudaSuccess) return GBDLT_ERR_CUDA;
  count_launch((int)b.graph_kernels);
  st = move(b, b.stage_out, out, false);
  if (st) return st;
  if (cudaEventRecord(b.ev_out, b.s) != cudaSuccess || cudaStreamWaitEvent(user, b.ev_out, 0) != cudaSuccess)
    return GBDLT_ERR_CUDA;
  return GBDLT_OK;
}

extern "C" int gbdlt_batch_info(gbdlt_batch batch, int64_t* total_elements, int64_t* groups,
                                int64_t* graph_kernels) {
  if (!batch) return GBDLT_ERR_INVALID_ARG;
  Batch& b = *reinterpret_cast<Batch*>(batch);
  if (total_elements) *total_elements = b.total;
  if (groups) *groups = (int64_t)b.groups.size();
  if (graph_kernels) *graph_kernels = b.graph_kernels;
  return GBDLT_OK;
}

extern "C" int gbdlt_batch_destroy(gbdlt_batch batch) {
  if (!batch) return GBDLT_ERR_INVALID_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  cudaStreamSynchronize(b->s);
  free_batch(b);
  return GBDLT_OK;
}
