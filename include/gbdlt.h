/*
 * gbdlt: fast discrete Legendre transform on one GPU (GB300, sm_103a).
 *
 * The method is Hale & Townsend, "A fast FFT-based discrete Legendre
 * transform": the DLT of Eq. (1) is computed as a Legendre -> Chebyshev
 * coefficient conversion (Sec. 3; asymptotic expansion of P_n(cos theta) summed
 * by DCT/DST over theta-bands, three-term recurrence where the expansion is not
 * accurate) followed by the non-uniform DCT of Sec. 2 (Taylor series in
 * delta-theta_k = theta^leg_k - theta^cheb1_k, each term one DCT or DST, Eq. 13).
 * The IDLT of Eq. (2) is the transposed chain of Sec. 4,
 * c = D_s M^T T_N^T(x^leg) D_w f with s_n = n + 1/2.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: GBDLT_OK (0) or a negative code.
 *   - Pointers to vector data are DEVICE pointers unless a name says "host".
 *     Data vectors are contiguous, [batch][N] row-major, element type given by
 *     the plan precision: double for GBDLT_FP64, float for GBDLT_FP32.  Node
 *     and weight arrays are always double.  Device data pointers must be
 *     aligned to their element size (8 bytes for double, 4 for float).
 *   - Inputs and outputs must not overlap unless a function says otherwise.
 *   - batch == 0 is a no-op that returns GBDLT_OK without reading the data
 *     pointers (they may be NULL); batch < 0 or a NULL data pointer with
 *     batch > 0 returns GBDLT_ERR_INVALID_ARG.
 *   - All work is enqueued on the plan's CUDA stream and is asynchronous; the
 *     caller owns every input/output buffer, the plan owns its node cache,
 *     tables and workspace.  gbdlt_plan_sync() waits for the stream and reports
 *     device-side failures (for instance a node iteration that did not settle).
 *     FP64 plans run the float-float and FP32 transforms of a stage on a
 *     plan-owned side stream that is forked from and joined back into the plan
 *     stream within the call, so a call's work stays ordered on the plan stream
 *     (inside a stream capture the side stream becomes a branch of the graph).
 *   - N is the transform length, 1 <= N <= 2^24: a power of two for the
 *     FFT-based chain, any N <= 65536 for the direct method (see
 *     GBDLT_METHOD_*).  Other N make plan creation return
 *     GBDLT_ERR_UNSUPPORTED_N.
 *   - A plan is not thread-safe: calls on one plan must be serialised.
 */
#ifndef GBDLT_H
#define GBDLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbdlt_plan_s* gbdlt_plan;

/* Arithmetic form.  GBDLT_FP64: double data in/out and FP64 accuracy: the
 * nodes, the recurrence region, the head block and the leading expansion and
 * Taylor terms in double; the terms whose size bounds their rounding error
 * within eps/20 (gbdlt_params M_ff, M_fp32, L_ff) have their transforms and
 * combines in float-float or FP32 arithmetic, scaled by exact powers of two.
 * GBDLT_FP32: DCT/DST transforms, asymptotic and Taylor combines in float; the
 * recurrence region in float-float (compensated float, ~2^-44 per operation)
 * with compensated sums; nodes, weights and delta-theta are computed in double.
 * Float data in/out. */
enum { GBDLT_FP64 = 0, GBDLT_FP32 = 1 };

enum {
  GBDLT_OK = 0,
  GBDLT_ERR_INVALID_ARG = -1,    /* null pointer, batch < 0, bad precision, ... */
  GBDLT_ERR_UNSUPPORTED_N = -2,  /* N out of range for the method asked for    */
  GBDLT_ERR_CUDA = -3,           /* a CUDA runtime call failed                */
  GBDLT_ERR_OOM = -4,            /* device allocation failed                  */
  GBDLT_ERR_NOT_CONVERGED = -5,  /* a node Newton iteration did not settle    */
  GBDLT_ERR_UNIMPLEMENTED = -6
};

/* How a plan computes gbdlt_dlt, gbdlt_idlt and their transposes.
 * GBDLT_METHOD_FAST: the FFT-based chain of Sec. 2-4.  For N a power of two it
 *   runs on the N-point Chebyshev grid; for other N on the grid of the next
 *   power of two G (gbdlt_params.grid_n): coefficient vectors are zero-padded
 *   to G, the rows are the N-point Gauss-Legendre rule, each row's Taylor
 *   expansion (Sec. 2.1-2.3) is taken about its nearest grid point, and L
 *   follows from Corollary 2.4 with |n dtheta| <= (N-1) pi / (2G) in place of
 *   0.83845; the cost is close to that of a plan for G.
 * GBDLT_METHOD_DIRECT: the O(N^2) sums of Eq. (1) and (2) evaluated by the
 *   three-term recurrence at the Legendre nodes (any N <= 65536); the direct
 *   approach the paper compares against, and faster on GB300 for small N.
 * GBDLT_METHOD_AUTO: DIRECT when N <= 256, FAST otherwise.  leg2cheb and
 *   chebeval always run the FFT-based chain (a DIRECT plan whose N is not a
 *   power of two has none: GBDLT_ERR_UNSUPPORTED_N). */
enum { GBDLT_METHOD_AUTO = 0, GBDLT_METHOD_FAST = 1, GBDLT_METHOD_DIRECT = 2 };

/* Parameters the plan derives from (N, precision, eps) by the error bounds of
 * the paper (Table 1 / Corollary 2.4 for L) and of the asymptotic expansion of
 * P_n(cos theta) (band cuts), choosing the cheapest feasible band layout. */
#define GBDLT_MAX_BANDS 32
typedef struct {
  int64_t N;
  int prec;
  double eps;          /* target max|error| / ||c||_1                          */
  int L;               /* Taylor terms (l = 0..L-1), Corollary 2.4             */
  int M;               /* terms of the asymptotic expansion of P_n(cos theta)  */
  int K;               /* number of theta-bands using the expansion            */
  int64_t band_ns[GBDLT_MAX_BANDS]; /* column cut: band b uses n >= band_ns[b]  */
  int64_t band_ka[GBDLT_MAX_BANDS]; /* rows [ka, kb) and [N-kb, N-ka)          */
  int64_t band_kb[GBDLT_MAX_BANDS];
  int64_t rec_steps;   /* recurrence (row, n) pairs, both halves              */
  int seg_len;         /* recurrence segment length of the fast path (512; 256 in FP32 plans) */
  double flops_dlt;    /* modelled arithmetic per DLT (flop)                  */
  double bytes_dlt;    /* algorithmic HBM bytes per DLT: read c, dtheta; write f */
  double bytes_idlt;   /* same for the IDLT (adds the weights)                */
  size_t workspace_bytes; /* device workspace the plan allocates              */
  int method;          /* GBDLT_METHOD_FAST or GBDLT_METHOD_DIRECT (resolved)  */
  int64_t direct_steps; /* half-row recurrence steps of one direct transform   */
  int64_t head;        /* fast path: columns n < head come from the dense block
                          M[0:head, 0:head] (Sec. 3); 0 = none                 */
  int M_fp32;          /* FP64 plans: the last M_fp32 expansion terms have their
                          band FFTs in FP32 (their size bounds the error)       */
  int M_ff;            /* FP64 plans: the M_ff terms before those run their band
                          FFTs in float-float arithmetic (FP32 pipe)            */
  int L_ff;            /* FP64 plans: the last L_ff Taylor terms run their FFTs
                          and combines in float-float                           */
  int64_t grid_n;      /* fast path: length of the Chebyshev grid and of its FFTs
                          (N for a power of two, else the next power of two);
                          0 for a DIRECT plan with N not a power of two        */
} gbdlt_params;

/* Host-only parameter derivation: no GPU, no allocation.  eps <= 0 selects the
 * default (1e-14 for GBDLT_FP64, 2e-6 for GBDLT_FP32).  Returns
 * GBDLT_ERR_UNSUPPORTED_N or GBDLT_ERR_INVALID_ARG on bad input. */
int gbdlt_plan_params(int64_t N, int prec, double eps, gbdlt_params* out);
/* The same for a given method (GBDLT_METHOD_*); GBDLT_ERR_UNSUPPORTED_N if N
 * does not suit it (N outside 1..2^24; DIRECT: N > 65536). */
int gbdlt_plan_params_ex(int64_t N, int prec, double eps, int method, gbdlt_params* out);

/* Create a plan on the current CUDA device.  `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream).  Computes the Legendre nodes and weights
 * (gbdlt_legpts), the per-N tables and allocates the workspace in one device
 * allocation (gbdlt_plan_get_params reports its size: FP64 plans with a head
 * block of h <= 32768 columns include its h^2/4 stored products twice, ordered
 * by rows and by columns, 1.07 GB at N = 2^20 and 4.3 GB at 2^22).  On error
 * *out is set to NULL and nothing is leaked. */
int gbdlt_plan_create(int64_t N, int prec, double eps, void* cuda_stream, gbdlt_plan* out);
/* gbdlt_plan_create with the method given (GBDLT_METHOD_AUTO is what
 * gbdlt_plan_create uses). */
int gbdlt_plan_create_ex(int64_t N, int prec, double eps, int method, void* cuda_stream, gbdlt_plan* out);
int gbdlt_plan_destroy(gbdlt_plan plan);
/* Change the stream later calls enqueue on. */
int gbdlt_plan_set_stream(gbdlt_plan plan, void* cuda_stream);
/* Wait for the plan's stream; returns GBDLT_ERR_NOT_CONVERGED if a node
 * iteration failed since the last sync, GBDLT_ERR_CUDA on a CUDA error. */
int gbdlt_plan_sync(gbdlt_plan plan);
int gbdlt_plan_get_params(gbdlt_plan plan, gbdlt_params* out);
/* Newton iterations a node may take in this plan's later gbdlt_legpts calls
 * (0 <= max_iter <= 24, the default and the largest value; the node solve of
 * Sec. 2.2 settles in 2-4).  A node that has not settled within the cap is
 * flagged and the next gbdlt_plan_sync returns GBDLT_ERR_NOT_CONVERGED (and
 * clears the flag); its theta, x, w and dtheta are then unspecified until a
 * gbdlt_legpts with a sufficient cap recomputes them.  A failure-path hook: it
 * lets a caller or a test reach the not-converged status without a fault.
 * GBDLT_ERR_INVALID_ARG for other values. */
int gbdlt_plan_set_node_iterations(gbdlt_plan plan, int max_iter);
/* How the plan's FP32 FFT passes (the FP32 form's transforms, and the FP32
 * tier of FP64 plans) move their tiles: enable = 1 uses the persistent passes
 * that copy each tile into shared memory with the tensor memory accelerator
 * while the previous tile is transformed (Remark 2.2's FFTs; column passes for
 * 2^13 <= N <= 2^23, row passes for N <= 2^21), enable = 0 the passes in which
 * every thread loads its part of the tile itself.  Default: 1 for GBDLT_FP32
 * plans with 2^18 <= N <= 2^21, where the whole DLT + IDLT measured faster
 * with it; 0 otherwise (neutral at smaller N, slower where the persistent
 * grid keeps kernels of the plan's side stream, or the FP64 kernels beside an
 * FP64 plan's FP32 transforms, off the SMs).  Both compute the same butterflies in the same
 * order, so results are bitwise identical; the choice only changes speed.
 * Clears the plan's replayed graphs.  GBDLT_ERR_INVALID_ARG for other values.
 * A staged copy that has not landed after about two seconds makes the next
 * gbdlt_plan_sync return GBDLT_ERR_CUDA. */
int gbdlt_plan_set_fft_staging(gbdlt_plan plan, int enable);
/* FP64 plans: run the FP64 and the float-float FFTs of each Taylor stage in one
 * pair of launches whose thread blocks alternate between the two kinds, so that
 * an SM holds one of each and both of GB300's FP64 and FP32 pipes work, or as
 * two launches on two streams.  mode 0: always two streams; 1 (the default):
 * mixed launches at N >= 2^20 (the plan's grid length), where they are faster,
 * two streams below; 2: mixed launches at every length above 4096.  The
 * butterflies are the same either way, so results are bitwise identical; the
 * choice only changes speed.  Clears the plan's replayed graphs.
 * GBDLT_ERR_INVALID_ARG for other values. */
int gbdlt_plan_set_fft_mix(gbdlt_plan plan, int mode);
/* SM clock cycles a staged FFT pass of this plan waits for a tile copy before
 * it gives up (0 <= sm_cycles <= 2^32; default 2^32, about two seconds).  A pass
 * that gives up records it (the next gbdlt_plan_sync returns GBDLT_ERR_CUDA and
 * clears the record), waits once more with the default limit for its own copy
 * in flight, and ends without finishing its tiles (that call's results are
 * unspecified).  A failure-path hook: a small limit reaches this status with no
 * fault.  Clears the plan's replayed graphs.  GBDLT_ERR_INVALID_ARG for other
 * values. */
int gbdlt_plan_set_wait_limit(gbdlt_plan plan, int64_t sm_cycles);

/* Legendre nodes and weights (Eq. 1 and Eq. 2; Sec. 2.1-2.2): recomputes the
 * plan's node cache on the GPU and copies any requested array out.  Ordering:
 * theta ascending, x = cos(theta) descending (1 > x_0 > ... > x_{N-1} > -1).
 * Outputs (device, N doubles each, any may be NULL): x, theta, w (Gauss-Legendre
 * weights), dtheta = theta_k - (k+1/2)pi/N (offset from the Chebyshev points of
 * the first kind, Eq. 5).  With every output NULL the recomputation is deferred
 * to the next call on this plan that reads the nodes: the FFT-based transforms
 * of a power-of-two plan run it as a branch beside their first stages (which do
 * not read the nodes) and wait for it before the Taylor step; other calls run it
 * first; gbdlt_plan_sync runs a refresh still pending, so its status (e.g.
 * GBDLT_ERR_NOT_CONVERGED) is reported there.  The nodes are the same either
 * way. */
int gbdlt_legpts(gbdlt_plan plan, double* x, double* theta, double* w, double* dtheta);

/* Allocation-free Gauss-Legendre rule, for callers that cannot call
 * cudaMalloc (a fixed pre-reserved memory budget owned by their own
 * allocator, a latency-critical path that cannot afford cudaMalloc's implicit
 * synchronisation, a plugin handed its buffers by a host framework).  The paper
 * has no counterpart; it is the node kernel of gbdlt_legpts without a plan.
 *   N: any integer 1 <= N <= 65536; larger N returns GBDLT_ERR_UNSUPPORTED_N.
 *   x, theta, w (device, N doubles each, required) and dtheta (device, N
 *   doubles, may be NULL): the same arrays and ordering as gbdlt_legpts.
 *   cuda_stream: cudaStream_t to run on (NULL = legacy default stream).
 * Allocates no memory (gbdlt_device_alloc_count does not change).  Its scratch
 * (N doubles and a status word) is a 512 KB array in the library's device
 * memory, present on every GPU that loads the library until the process exits.
 * Every call looks up that array's device address in the current device's
 * context (the first call on a device may load the library's device code there:
 * make that first call before any stream capture on that device); a call after
 * cudaDeviceReset therefore uses the array of the new context.  Every call uses
 * the same array, so calls that overlap on the GPU (different streams,
 * different host threads) race and must be serialised by the caller.
 * Synchronises `cuda_stream` before returning and returns
 * GBDLT_ERR_NOT_CONVERGED if a node iteration did not settle. */
int gbdlt_legpts_noalloc(int64_t N, double* x, double* theta, double* w, double* dtheta,
                         void* cuda_stream);

/* Legendre -> Chebyshev coefficients (Sec. 3): chat = M c. */
int gbdlt_leg2cheb(gbdlt_plan plan, const void* c, void* chat, int64_t batch);
/* Transpose: out = M^T y (Sec. 4, item 3). */
int gbdlt_leg2cheb_t(gbdlt_plan plan, const void* y, void* out, int64_t batch);
/* Chebyshev expansion evaluated at the Legendre nodes, Eq. (3) (the NDCT of
 * Sec. 2): f_k = sum_n chat_n T_n(x^leg_k). */
int gbdlt_chebeval(gbdlt_plan plan, const void* chat, void* f, int64_t batch);
/* Transpose (Sec. 4, item 2): out_n = sum_k g_k T_n(x^leg_k). */
int gbdlt_chebeval_t(gbdlt_plan plan, const void* g, void* out, int64_t batch);
/* DLT, Eq. (1): f_k = sum_n c_n P_n(x^leg_k). */
int gbdlt_dlt(gbdlt_plan plan, const void* c, void* f, int64_t batch);
/* Transposed DLT (Sec. 4): out_n = sum_k g_k P_n(x^leg_k). */
int gbdlt_dlt_t(gbdlt_plan plan, const void* g, void* out, int64_t batch);
/* IDLT, Eq. (2): c_n = (n + 1/2) sum_k w_k f_k P_n(x^leg_k). */
int gbdlt_idlt(gbdlt_plan plan, const void* f, void* c, int64_t batch);
/* Transposed IDLT: out = D_w P_N(x^leg) D_s g, i.e. out_k = w_k sum_n (n+1/2) g_n P_n(x_k). */
int gbdlt_idlt_t(gbdlt_plan plan, const void* g, void* out, int64_t batch);

/* Uneven batches (no counterpart in the paper, which transforms one vector at
 * a time): B transforms of lengths Ns_host[i] (1..2^24) and directions dirs_host[i]
 * (0 = DLT, 1 = IDLT), all of one precision, executed together.  Inputs and
 * outputs are concatenated in the given order: transform i occupies elements
 * [sum_{j<i} Ns[j], sum_{j<=i} Ns[j]) of `in` and `out` (device, element type
 * of `prec`).  Creation buckets the transforms by (G, direction), G the power
 * of two with G/2 < N <= G.  A bucket of one length is one group (N, direction)
 * with its own plan.  A bucket of several lengths is one grid group (one chain
 * on the grid G for all its transforms, each with its own N-point rule; see
 * GBDLT_METHOD_FAST) or, under DIRECT (or AUTO with G <= 512), one direct group
 * per length.  Every group's plan is sized for the whole group; creation spreads the
 * groups over up to 8 internal
 * streams, picks each group's method and captures every group's batched chain
 * into one CUDA graph with one branch per stream (1 <= B <= 65535).  With
 * GBDLT_METHOD_AUTO the method of a group that allows both is chosen by timing
 * both on the device at creation (the autotuner; see gbdlt_batch_group_info),
 * so two batch objects over the same lengths may choose differently; FAST or
 * DIRECT force one method (GBDLT_ERR_UNSUPPORTED_N where a length does not suit
 * it).  An execution makes the work wait for `cuda_stream`, gathers `in` into
 * the staging buffers, replays the graph, scatters the results into `out` and
 * makes `cuda_stream` wait for them; it allocates nothing.  Executions of one
 * batch object must not overlap.  Direct-method groups whose transforms each
 * fit one thread block (N <= 512) do not get a chain of their own: all such
 * transforms of one direction run in a single persistent launch that strides
 * over a job table fixed at creation (longest transforms first), with results
 * bitwise those of the group's single-plan calls.  gbdlt_batch_create =
 * gbdlt_batch_create_ex with GBDLT_METHOD_AUTO. */
typedef struct gbdlt_batch_s* gbdlt_batch;
int gbdlt_batch_create(const int64_t* Ns_host, const int32_t* dirs_host, int64_t B, int prec,
                       double eps, gbdlt_batch* out);
int gbdlt_batch_create_ex(const int64_t* Ns_host, const int32_t* dirs_host, int64_t B, int prec,
                          double eps, int method, gbdlt_batch* out);
int gbdlt_batch_exec(gbdlt_batch batch, const void* in, void* out, void* cuda_stream);
/* Group g (0 <= g < groups, in staging order): its length, direction, number of
 * transforms, the method it runs, and the autotuner's milliseconds per run of
 * the whole group by each method (-1 where that method was not timed).  Any
 * output pointer may be NULL. */
int gbdlt_batch_group_info(gbdlt_batch batch, int64_t g, int64_t* N, int32_t* dir, int64_t* count,
                           int32_t* method, double* ms_fast, double* ms_direct);
/* As gbdlt_batch_group_info, and *fused = 1 where the group runs inside its
 * direction's persistent direct launch, else 0; *lengths = the number of
 * distinct lengths the group holds (1, or for a grid group, whose *N is the grid
 * G, its lengths in (G/2, G]). */
int gbdlt_batch_group_info_ex(gbdlt_batch batch, int64_t g, int64_t* N, int32_t* dir, int64_t* count,
                              int32_t* method, double* ms_fast, double* ms_direct, int32_t* fused,
                              int64_t* lengths);
/* total elements of the concatenated layout, number of (N, direction) groups,
 * kernel nodes in the captured graph (any pointer may be NULL) */
int gbdlt_batch_info(gbdlt_batch batch, int64_t* total_elements, int64_t* groups,
                     int64_t* graph_kernels);
int gbdlt_batch_destroy(gbdlt_batch batch);

/* Per-kernel device timing on the plan's stream, for profiling (off by
 * default).  mode 1: turn on and start timing from this point (work enqueued
 * earlier is not attributed); call again before each region to re-anchor.
 * mode 0: turn off.  mode 2: clear the accumulated totals.  While on, the
 * library records one CUDA event after every kernel it launches. */
int gbdlt_plan_profile(gbdlt_plan plan, int mode);
/* Report of the accumulated timing: one line per kernel,
 * "name launches total_ms flops bytes", where flops and bytes are the
 * algorithmic counts of those launches.  Waits for the recorded events.
 * Writes at most len-1 characters and a NUL into buf (buf may be NULL when
 * len == 0); returns the length of the full report, or a negative status. */
int64_t gbdlt_plan_profile_read(gbdlt_plan plan, char* buf, int64_t len);

/* Human-readable name of a status code (static string). */
const char* gbdlt_status_string(int status);
/* Number of kernels this library has launched since it was loaded (all plans,
 * all threads). */
uint64_t gbdlt_launch_count(void);
/* Number of device allocations (cudaMalloc calls) this library has made since
 * it was loaded: plan workspaces, plan-creation scratch and batch staging
 * buffers (all plans and batches, all threads). */
uint64_t gbdlt_device_alloc_count(void);
/* Measurement helper (no counterpart in the paper): the FP64 arithmetic rate
 * this device reaches, the denominator of the roofline of the FP64 kernels,
 * whose bound is the FP64 pipe.  Runs a kernel of independent FP64 fused
 * multiply-add chains (8 per thread, 8 CTAs of 256 threads per SM, a fixed
 * loop count) four times on `cuda_stream` (a cudaStream_t, NULL = legacy
 * default) and stores 2 flops per FMA divided by the fastest of the last three
 * runs (CUDA events) into *flops_per_second.  Synchronises the stream; makes
 * one small device allocation.  GBDLT_ERR_INVALID_ARG for a null pointer,
 * GBDLT_ERR_CUDA / GBDLT_ERR_OOM on a runtime failure. */
int gbdlt_fp64_fma_rate(void* cuda_stream, double* flops_per_second);

#ifdef __cplusplus
}
#endif
#endif /* GBDLT_H */
