// Uneven batches: many transforms of different lengths and directions run as
// one CUDA-graph replay.
//
// The transforms are grouped by (N, direction).  Each group gets its own plan,
// whose workspace holds the whole group in one pass, so a group is a single
// batched chain (every kernel carries the batch index in blockIdx.y and every
// FFT launch transforms all vectors of the group).  Groups are spread over up to
// kLanes internal streams, so that the graph has independent branches and small
// groups run side by side.
//
// Method per group (the autotuner): with GBDLT_METHOD_AUTO, a group whose N
// allows both methods is run and timed with CUDA events through the FFT-based
// chain and through the direct method (three timed runs each after a warm-up
// run) and keeps the faster; lengths above the direct method's limit take the
// FFT-based chain (on the next power-of-two grid when N is not a power of two).  The timings are kept and
// reported by gbdlt_batch_group_info.
//
// At creation the chains are run once more with the chosen methods and then
// captured from the internal streams into one CUDA graph (fork from the main
// internal stream, one branch per lane, join).  An execution is: wait for the
// caller's stream, gather the caller's concatenated inputs into the grouped
// staging layout, replay the graph, scatter the grouped outputs back to the
// caller's layout, and make the caller's stream wait for the result.  Nothing is
// allocated per execution.
#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "gbdlt_internal.cuh"

namespace gbdlt {

constexpr int kLanes = 8;
// buckets of several lengths with G up to this run the direct method under AUTO
// (the fused persistent launch; per-length timings favour it up to N = 512)
constexpr int64_t kBatchDirectG = 512;

struct BatchGroup {
  int64_t N;
  int dir;  // 0: DLT, 1: IDLT
  int64_t count;
  int64_t stage_off;  // element offset of the group's first vector in the staging buffers
  Plan* plan;
  int lane;           // internal stream the group runs on
  int method;         // GBDLT_METHOD_FAST or GBDLT_METHOD_DIRECT
  double ms_fast = -1.0, ms_direct = -1.0;  // autotuner timings (-1: not timed)
  bool fused = false;  // runs inside the direction's persistent direct launch
  int64_t stride = 0;  // staging elements per transform: N, or G for a grid group
  int64_t lengths = 1; // distinct lengths (a grid group's rules)
  GridRules* rules = nullptr;  // grid group: the rule of every length
  int32_t* d_item = nullptr;   // grid group: rule of each item (device)
};

struct Batch {
  int prec = GBDLT_FP64;
  int64_t B = 0, total = 0, maxN = 0;
  int64_t stage_total = 0;  // staging elements (grid groups take G per transform)
  cudaStream_t s = nullptr;
  cudaStream_t lane_s[kLanes] = {};
  cudaEvent_t lane_ev[kLanes] = {};
  cudaEvent_t ev_fork = nullptr;
  int nlanes = 0;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<Plan*> plans;
  std::vector<BatchGroup> groups;
  int64_t* d_src = nullptr;    // [B] offset of transform i in the caller's layout
  int64_t* d_stage = nullptr;  // [B] offset of transform i in the staging layout
  int64_t* d_len = nullptr;    // [B] N_i
  void* stage_in = nullptr;
  void* stage_out = nullptr;
  DirectMulti* direct[2] = {};  // persistent direct launches (DLT, IDLT) over the small groups
  int direct_lane[2] = {};
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

int run_group(Batch& b, const BatchGroup& g, int method) {
  const size_t es = b.prec == GBDLT_FP64 ? 8 : 4;
  const char* in = (const char*)b.stage_in + (size_t)g.stage_off * es;
  char* out = (char*)b.stage_out + (size_t)g.stage_off * es;
  return run_op_method(reinterpret_cast<gbdlt_plan>(g.plan), g.dir ? OP_IDLT : OP_DLT, method, in, out, g.count);
}

// every group on its lane: the lanes wait for b.s, then b.s waits for the lanes
int run_groups(Batch& b) {
  if (cudaEventRecord(b.ev_fork, b.s) != cudaSuccess) return GBDLT_ERR_CUDA;
  for (int l = 0; l < b.nlanes; ++l)
    if (cudaStreamWaitEvent(b.lane_s[l], b.ev_fork, 0) != cudaSuccess) return GBDLT_ERR_CUDA;
  for (int d = 0; d < 2; ++d) {
    int st = direct_multi_launch(b.direct[d], b.lane_s[b.direct_lane[d]]);
    if (st) return st;
  }
  for (const BatchGroup& g : b.groups) {
    if (g.fused) continue;
    int st = run_group(b, g, g.method);
    if (st) return st;
  }
  for (int l = 0; l < b.nlanes; ++l) {
    if (cudaEventRecord(b.lane_ev[l], b.lane_s[l]) != cudaSuccess) return GBDLT_ERR_CUDA;
    if (cudaStreamWaitEvent(b.s, b.lane_ev[l], 0) != cudaSuccess) return GBDLT_ERR_CUDA;
  }
  return GBDLT_OK;
}

// milliseconds per run of group g with `method`: one warm-up run, three timed
double time_group(Batch& b, BatchGroup& g, int method, cudaEvent_t e0, cudaEvent_t e1, int* status) {
  cudaStream_t st = b.lane_s[g.lane];
  *status = run_group(b, g, method);
  if (*status) return -1.0;
  if (cudaEventRecord(e0, st) != cudaSuccess) {
    *status = GBDLT_ERR_CUDA;
    return -1.0;
  }
  for (int r = 0; r < 3 && !*status; ++r) *status = run_group(b, g, method);
  if (*status) return -1.0;
  float ms = 0.f;
  if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
    *status = GBDLT_ERR_CUDA;
    return -1.0;
  }
  return (double)ms / 3.0;
}

void free_batch(Batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (DirectMulti* d : b->direct) direct_multi_free(d);
  for (Plan* p : b->plans) free_plan(p);
  for (BatchGroup& g : b->groups) {
    if (g.rules) grid_rules_free(g.rules);
    if (g.d_item) cudaFree(g.d_item);
  }
  if (b->d_src) cudaFree(b->d_src);
  if (b->stage_in) cudaFree(b->stage_in);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (int l = 0; l < kLanes; ++l) {
    if (b->lane_ev[l]) cudaEventDestroy(b->lane_ev[l]);
    if (b->lane_s[l]) cudaStreamDestroy(b->lane_s[l]);
  }
  if (b->s) cudaStreamDestroy(b->s);
  delete b;
}

}  // namespace

}  // namespace gbdlt

using namespace gbdlt;

struct gbdlt_batch_s {};  // opaque tag; the pointer is a gbdlt::Batch

extern "C" int gbdlt_batch_create_ex(const int64_t* Ns_host, const int32_t* dirs_host, int64_t B, int prec,
                                     double eps, int method, gbdlt_batch* out) {
  if (!out) return GBDLT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!Ns_host || !dirs_host || B < 1 || B > 65535) return GBDLT_ERR_INVALID_ARG;
  if (prec != GBDLT_FP64 && prec != GBDLT_FP32) return GBDLT_ERR_INVALID_ARG;
  if (method != GBDLT_METHOD_AUTO && method != GBDLT_METHOD_FAST && method != GBDLT_METHOD_DIRECT)
    return GBDLT_ERR_INVALID_ARG;
  for (int64_t i = 0; i < B; ++i) {
    const int64_t N = Ns_host[i];
    if (N < 1 || N > (1ll << 24)) return GBDLT_ERR_UNSUPPORTED_N;
    if (method == GBDLT_METHOD_DIRECT && N > kDirectMax) return GBDLT_ERR_UNSUPPORTED_N;
    if (dirs_host[i] != 0 && dirs_host[i] != 1) return GBDLT_ERR_INVALID_ARG;
  }
  Batch* b = new (std::nothrow) Batch();
  if (!b) return GBDLT_ERR_OOM;
  b->prec = prec;
  b->B = B;
  const size_t es = prec == GBDLT_FP64 ? 8 : 4;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  auto fail = [&](int st) {
    cudaGetLastError();
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    free_batch(b);
    return st;
  };
  if (cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess)
    return fail(GBDLT_ERR_CUDA);
  // Groups.  Transforms are bucketed by (G, dir), G the power of two with
  // G/2 < N <= G.  A bucket of one length is one group (N, dir) as it stands.
  // A bucket of several lengths is either one grid group (one chain on the grid
  // G for all its transforms, each item with its own rule: grid.cu), or, under
  // the direct method (forced, or AUTO with G <= kBatchDirectG, where the
  // per-length autotuner timings favoured it), one direct group per length.
  std::map<std::pair<int64_t, int>, std::vector<int64_t>> buckets;
  std::vector<int64_t> src(B), stage(B), len(B);
  int64_t off = 0;
  for (int64_t i = 0; i < B; ++i) {
    src[i] = off;
    len[i] = Ns_host[i];
    off += Ns_host[i];
    b->maxN = std::max(b->maxN, Ns_host[i]);
    int64_t G = 1;
    while (G < Ns_host[i]) G <<= 1;
    buckets[{G, dirs_host[i]}].push_back(i);
  }
  b->total = off;
  struct Proto {
    int64_t N, G;
    int dir;
    bool grid;
    std::vector<int64_t> idx;
  };
  std::vector<Proto> protos;
  for (auto& kv : buckets) {
    const int64_t G = kv.first.first;
    const int dir = kv.first.second;
    std::map<int64_t, std::vector<int64_t>> byN;
    for (int64_t i : kv.second) byN[Ns_host[i]].push_back(i);
    const bool direct = method == GBDLT_METHOD_DIRECT || (method == GBDLT_METHOD_AUTO && G <= kBatchDirectG);
    if (byN.size() > 1 && !direct) {
      protos.push_back(Proto{G, G, dir, true, kv.second});
    } else {
      for (auto& nv : byN) protos.push_back(Proto{nv.first, G, dir, false, nv.second});
    }
  }
  b->nlanes = (int)std::min<size_t>(kLanes, protos.size());
  for (int l = 0; l < b->nlanes; ++l)
    if (cudaStreamCreateWithFlags(&b->lane_s[l], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->lane_ev[l], cudaEventDisableTiming) != cudaSuccess)
      return fail(GBDLT_ERR_CUDA);
  // one plan per group, on the group's lane; groups go to lanes in order of
  // decreasing work so that the lanes carry similar loads
  std::vector<std::pair<double, size_t>> order;
  for (size_t q = 0; q < protos.size(); ++q)
    order.push_back({-(double)protos[q].idx.size() * (double)(protos[q].grid ? protos[q].G : protos[q].N), q});
  std::sort(order.begin(), order.end());
  std::vector<double> lane_load(b->nlanes, 0.0);
  int64_t soff = 0;
  for (auto& ok : order) {
    const Proto& pr = protos[ok.second];
    const std::vector<int64_t>& idx = pr.idx;
    BatchGroup g;
    g.N = pr.N;
    g.dir = pr.dir;
    g.count = (int64_t)idx.size();
    g.stage_off = soff;
    g.stride = pr.N;
    g.lane = (int)(std::min_element(lane_load.begin(), lane_load.end()) - lane_load.begin());
    lane_load[g.lane] += -ok.first;
    Plan* p = nullptr;
    if (pr.grid) {
      // one node plan per length (its rule), the chain of a plan for G
      std::map<int64_t, int32_t> rule_of;
      std::vector<Plan*> nodes;
      double bmax = 0.0;
      for (int64_t i : idx) {
        if (rule_of.count(Ns_host[i])) continue;
        Plan* np = nullptr;
        int st = plan_create_nodes(Ns_host[i], prec, b->lane_s[g.lane], &np);
        if (st) return fail(st);
        b->plans.push_back(np);
        rule_of[Ns_host[i]] = (int32_t)nodes.size();
        nodes.push_back(np);
        bmax = std::max(bmax, grid_bound(Ns_host[i], pr.G));
      }
      int st = plan_create_grid(pr.G, prec, eps, bmax, b->lane_s[g.lane], g.count, &p);
      if (st) return fail(st);
      b->plans.push_back(p);
      st = grid_rules_create(pr.G, nodes, b->lane_s[g.lane], &g.rules);
      if (st) return fail(st);
      std::vector<int32_t> item(idx.size());
      for (size_t q = 0; q < idx.size(); ++q) item[q] = rule_of[Ns_host[idx[q]]];
      if (dev_malloc((void**)&g.d_item, sizeof(int32_t) * item.size()) != cudaSuccess ||
          cudaMemcpy(g.d_item, item.data(), sizeof(int32_t) * item.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        b->groups.push_back(g);  // freed with the batch
        return fail(GBDLT_ERR_CUDA);
      }
      st = grid_attach(*p, g.rules, g.d_item, false);
      if (st) {
        b->groups.push_back(g);
        return fail(st);
      }
      g.stride = pr.G;
      g.lengths = (int64_t)nodes.size();
      g.method = GBDLT_METHOD_FAST;
    } else {
      const bool can_direct = g.N > 1 && g.N <= kDirectMax;
      int m = method;
      if (m == GBDLT_METHOD_AUTO && !can_direct) m = GBDLT_METHOD_FAST;
      // several lengths of one bucket under AUTO: the direct method, untimed
      if (m == GBDLT_METHOD_AUTO && buckets[{pr.G, pr.dir}].size() != idx.size()) m = GBDLT_METHOD_DIRECT;
      const int plan_method = m == GBDLT_METHOD_AUTO ? GBDLT_METHOD_FAST : m;
      int st = plan_create_impl(g.N, prec, eps, plan_method, b->lane_s[g.lane], g.count,
                                m == GBDLT_METHOD_AUTO ? 1 : 0, &p);
      if (st) return fail(st);
      b->plans.push_back(p);
      g.method = m;  // AUTO is resolved by the timing below
    }
    g.plan = p;
    for (size_t q = 0; q < idx.size(); ++q) stage[idx[q]] = soff + (int64_t)q * g.stride;
    soff += g.count * g.stride;
    b->groups.push_back(g);
  }
  b->stage_total = soff;
  // device tables and staging (zeroed once: a grid group's slots keep zeros past
  // each transform's length, which the gather never writes)
  if (dev_malloc((void**)&b->d_src, sizeof(int64_t) * 3 * (size_t)B) != cudaSuccess) return fail(GBDLT_ERR_OOM);
  b->d_stage = b->d_src + B;
  b->d_len = b->d_src + 2 * B;
  if (dev_malloc((void**)&b->stage_in, 2 * es * (size_t)b->stage_total) != cudaSuccess) return fail(GBDLT_ERR_OOM);
  b->stage_out = (char*)b->stage_in + es * (size_t)b->stage_total;
  if (cudaMemcpy(b->d_src, src.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_stage, stage.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_len, len.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemsetAsync(b->stage_in, 0, 2 * es * (size_t)b->stage_total, b->s) != cudaSuccess ||
      cudaStreamSynchronize(b->s) != cudaSuccess)
    return fail(GBDLT_ERR_CUDA);
  // the autotuner: time both methods where both are open, keep the faster
  for (BatchGroup& g : b->groups) {
    if (g.method != GBDLT_METHOD_AUTO) continue;
    int st = GBDLT_OK;
    g.ms_fast = time_group(*b, g, GBDLT_METHOD_FAST, t0, t1, &st);
    if (st) return fail(st);
    g.ms_direct = time_group(*b, g, GBDLT_METHOD_DIRECT, t0, t1, &st);
    if (st) return fail(st);
    g.method = g.ms_direct < g.ms_fast ? GBDLT_METHOD_DIRECT : GBDLT_METHOD_FAST;
  }
  // direct-method groups whose transforms each fit one CTA run as one persistent
  // launch per direction, on the lane of the largest such group
  for (int d = 0; d < 2; ++d) {
    std::vector<DirectGroupRef> refs;
    int lane = -1;
    for (BatchGroup& g : b->groups) {
      if (g.dir != d || g.method != GBDLT_METHOD_DIRECT || !direct_fusable(*g.plan)) continue;
      refs.push_back({g.plan, g.count, (const char*)b->stage_in + (size_t)g.stage_off * es,
                      (char*)b->stage_out + (size_t)g.stage_off * es});
      g.fused = true;
      if (lane < 0) lane = g.lane;  // groups are in order of decreasing work
    }
    if (refs.empty()) continue;
    int st = direct_multi_create(refs, prec, d, &b->direct[d]);
    if (st) return fail(st);
    b->direct_lane[d] = lane;
  }
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
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  *out = reinterpret_cast<gbdlt_batch>(b);
  return GBDLT_OK;
}

extern "C" int gbdlt_batch_create(const int64_t* Ns_host, const int32_t* dirs_host, int64_t B, int prec,
                                  double eps, gbdlt_batch* out) {
  return gbdlt_batch_create_ex(Ns_host, dirs_host, B, prec, eps, GBDLT_METHOD_AUTO, out);
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

extern "C" int gbdlt_batch_group_info(gbdlt_batch batch, int64_t g, int64_t* N, int32_t* dir, int64_t* count,
                                      int32_t* method, double* ms_fast, double* ms_direct) {
  return gbdlt_batch_group_info_ex(batch, g, N, dir, count, method, ms_fast, ms_direct, nullptr, nullptr);
}

extern "C" int gbdlt_batch_group_info_ex(gbdlt_batch batch, int64_t g, int64_t* N, int32_t* dir, int64_t* count,
                                         int32_t* method, double* ms_fast, double* ms_direct, int32_t* fused,
                                         int64_t* lengths) {
  if (!batch) return GBDLT_ERR_INVALID_ARG;
  Batch& b = *reinterpret_cast<Batch*>(batch);
  if (g < 0 || g >= (int64_t)b.groups.size()) return GBDLT_ERR_INVALID_ARG;
  const BatchGroup& G = b.groups[(size_t)g];
  if (N) *N = G.N;
  if (dir) *dir = G.dir;
  if (count) *count = G.count;
  if (method) *method = G.method;
  if (ms_fast) *ms_fast = G.ms_fast;
  if (ms_direct) *ms_direct = G.ms_direct;
  if (fused) *fused = G.fused ? 1 : 0;
  if (lengths) *lengths = G.lengths;
  return GBDLT_OK;
}

extern "C" int gbdlt_batch_destroy(gbdlt_batch batch) {
  if (!batch) return GBDLT_ERR_INVALID_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  cudaStreamSynchronize(b->s);
  for (int l = 0; l < b->nlanes; ++l) cudaStreamSynchronize(b->lane_s[l]);
  free_batch(b);
  return GBDLT_OK;
}
