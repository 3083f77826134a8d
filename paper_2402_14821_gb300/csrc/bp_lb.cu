// bp_lb.cu -- C ABI of the DFF lower-bound feasibility check (include/bp_lb.h).
//
// Host side: argument checks, handle-owned scratch, launch configuration and
// the plain single-check path (one H2D copy, one kernel launch, one D2H copy,
// one synchronisation -- the shape of Alg. 3 with the six per-DFF launches
// merged into one).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <array>
#include <vector>

#include "../../include/bp_lb.h"
#include "bp_lb_core.cuh"
#include "bp_lb_eval.cuh"
#include "bp_lb_kernels.cuh"
#include "bp_lb_launch.cuh"
#include "bp_lb_l2.cuh"

using namespace bplb;

namespace {

constexpr size_t kListBytes = 2 * sizeof(uint32_t) * kListTop;  // items + fp32 quotients

constexpr int kModePlainRagged = 3;  // BP_MODE_PLAIN_RAGGED
constexpr int kModePlainNodes = 4;   // BP_MODE_PLAIN_NODES
constexpr int kPlainDefaultShape = 6;

struct PlainOut {  // device and pinned-host layout of one plain result
  int64_t bound;
  int64_t pad;
  bp_argmax_t arg;
  uint8_t feasible;
  uint8_t pad2[15];
};

}  // namespace

struct bp_lb {
  int device = 0;
  int num_sms = 0;
  int64_t capacity = 0;
  int64_t max_items = 0;
  cudaStream_t stream = nullptr;  // plain path
  // plain path
  int32_t *d_items = nullptr;
  int32_t *d_assign = nullptr;
  int32_t *h_items = nullptr;   // pinned
  int32_t *h_assign = nullptr;  // pinned
  PlainOut *d_out = nullptr;
  PlainOut *h_out = nullptr;    // pinned
  unsigned long long *d_key1 = nullptr;
  unsigned int *d_done1 = nullptr;
  // batch scratch
  int32_t cap_batch = 0;
  int64_t *d_tile_start = nullptr;
  int64_t *d_ptile_start = nullptr;  // prefix-kernel tile table
  int64_t *d_ctile_start = nullptr;  // cluster-kernel unit table
  int64_t *d_vtile_start = nullptr;  // VB2-kernel tile table
  int32_t prefix_on = 1;             // batched modes: BP_ALGO_PREFIX (default) or DIRECT
  int32_t plain_prefix_on = 1;       // plain modes
  // global-memory slices for prefix tables too large for shared memory:
  // kGlobalTableInts int32 per prefix-kernel CTA, allocated on first use
  int32_t *d_gscratch = nullptr;
  int64_t gscratch_ctas = 0;
  bool gscratch_failed = false;
  // tables too large for one CTA but within a cluster's shared memory go to
  // the cluster kernel (bp_lb_set_cluster_tables, or the batched autotuners;
  // default off); its resident clusters per launch, cached per mode and
  // shared-memory size
  int32_t cluster_on = 0;
  int cl_clusters[3] = {0, 0, 0};
  size_t cl_smem[3] = {0, 0, 0};
  // batched modes send VB2 (c <= 65535) to the VB2 kernel; the plain path
  // keeps it in the direct kernel (one launch fewer per check)
  int32_t vb2_on = 1;
  int32_t verdict = 0;  // BP_RESULT_FULL (0) or BP_RESULT_VERDICT (1)
  int32_t prune = 1;    // skip VB2 parameters that provably cannot win (exact)
  int32_t reduce_mode = BP_REDUCE_LOADS;     // search-node reduction variant
  const int64_t *d_bin_max_offsets = nullptr;  // optional per-bin maximum loads (caller's)
  const int32_t *d_bin_max = nullptr;
  // With prefix_ctas > 0, batched calls run the prefix-count kernel (then the
  // generic kernel) on a high-priority side stream beside the VB2 kernel:
  // prefix_ctas CTAs per SM for the prefix kernel, the rest of each SM for
  // VB2.  Default 0: one after another (faster on the search-node batch, the
  // latency-bound prefix kernel needs all its resident CTAs).
  int32_t prefix_ctas = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_cjoin = nullptr;  // the cluster kernel's end on the side stream
  uint32_t dff_off = 0;  // DFFs left out of the bound (bit d), default none
  // VB2's parameter cap of Sec. 4 (bp_lb_set_vb2_cap): off by default; when
  // on, vb2cap_kernel writes each instance's last VB2 parameter here
  int32_t vb2_cap = 0;
  int64_t *d_vb2hi = nullptr;   // [cap_batch], batched calls
  int64_t *d_vb2hi1 = nullptr;  // [1], the plain path
  // bp_lb_eval_range: its own result slot, ticket and (unused) outputs, so
  // that it never shares scratch with the plain path's stream
  unsigned long long *d_rkey = nullptr;
  unsigned int *d_rdone = nullptr;
  PlainOut *d_rout = nullptr;
  int64_t *d_rvb2hi = nullptr;
  // optional per-kernel timing of batched calls (events around each launch)
  bool timing = false;
  unsigned long long *d_work_count = nullptr;  // 4 counters (EvalArgs::work_count)
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::array<cudaEvent_t, 8>> ev_pending;
  size_t ev_next = 0;
  unsigned long long *d_keys = nullptr;
  unsigned int *d_done = nullptr;
  long long *d_isums = nullptr;  // [cap_batch][8] instance sums (EvalArgs::isums)
  unsigned long long *d_work = nullptr;
  // launch shape (index into kShapes) per mode: batched ragged i32, ragged
  // i64, nodes, then the plain ragged and plain node paths; occupancy cache of
  // the batched modes
  int shape[5] = {0, 0, 0, kPlainDefaultShape, kPlainDefaultShape};
  int occ_shape[3] = {-1, -1, -1};
  size_t occ_smem[3] = {0, 0, 0};
  int occ_blocks[3] = {0, 0, 0};
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BP_OK;
  if (e == cudaErrorMemoryAllocation) return BP_ENOMEM;
  return BP_ECUDA;
}

#define BP_CHECK(call)                        \
  do {                                        \
    const int _s = cuda_status(call);         \
    if (_s != BP_OK) return _s;               \
  } while (0)

#define BP_CHECK_STATUS(expr)                 \
  do {                                        \
    const int _s = (expr);                    \
    if (_s != BP_OK) return _s;               \
  } while (0)

template <int MODE>
size_t eval_smem(int64_t max_bins) {
  return kListBytes + (MODE == kSrcNodes ? sizeof(uint32_t) * (size_t)max_bins : 0);
}

// Resident CTAs per SM of the handle's shape for `mode` at `smem` bytes.
int occupancy(bp_lb *h, int mode, size_t smem) {
  const int s = h->shape[mode];
  if (h->occ_shape[mode] == s && h->occ_smem[mode] == smem) return h->occ_blocks[mode];
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, (const void *)eval_fn(s, mode),
                                                    kShapes[s].nt, smem) != cudaSuccess)
    return 0;
  h->occ_shape[mode] = s;
  h->occ_smem[mode] = smem;
  h->occ_blocks[mode] = blocks;
  return blocks;
}

// One launch of fn; with pdl, with programmatic stream serialization (the
// kernel may be scheduled while the previous one in the stream finishes, and
// waits for it itself: pdl_wait).
int launch_fn(const void *fn, unsigned grid, unsigned block, size_t smem, cudaStream_t st,
              EvalArgs &A, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1u : 0u;
  void *args[] = {&A};
  return cuda_status(cudaLaunchKernelExC(&cfg, fn, args));
}

int launch_eval(int shape, int mode, unsigned grid, size_t smem, cudaStream_t st, EvalArgs &A,
                bool pdl = false) {
  return launch_fn((const void *)eval_fn(shape, mode), grid, (unsigned)kShapes[shape].nt, smem, st,
                   A, pdl);
}

int grow_batch(bp_lb *h, int32_t B) {
  if (B <= h->cap_batch) return BP_OK;
  int32_t cap = std::max<int32_t>(B, 1024);
  cudaFree(h->d_tile_start);
  cudaFree(h->d_ptile_start);
  cudaFree(h->d_ctile_start);
  cudaFree(h->d_vtile_start);
  cudaFree(h->d_keys);
  cudaFree(h->d_done);
  cudaFree(h->d_isums);
  cudaFree(h->d_vb2hi);
  h->d_isums = nullptr;
  h->d_vb2hi = nullptr;
  h->d_tile_start = nullptr;
  h->d_ptile_start = nullptr;
  h->d_ctile_start = nullptr;
  h->d_vtile_start = nullptr;
  h->d_keys = nullptr;
  h->d_done = nullptr;
  h->cap_batch = 0;
  BP_CHECK(cudaMalloc(&h->d_tile_start, sizeof(int64_t) * ((size_t)cap + 1)));
  BP_CHECK(cudaMalloc(&h->d_ptile_start, sizeof(int64_t) * ((size_t)cap + 1)));
  BP_CHECK(cudaMalloc(&h->d_ctile_start, sizeof(int64_t) * ((size_t)cap + 1)));
  BP_CHECK(cudaMalloc(&h->d_vtile_start, sizeof(int64_t) * ((size_t)cap + 1)));
  BP_CHECK(cudaMalloc(&h->d_keys, sizeof(unsigned long long) * (size_t)cap));
  BP_CHECK(cudaMalloc(&h->d_done, sizeof(unsigned int) * (size_t)cap));
  BP_CHECK(cudaMalloc(&h->d_isums, sizeof(long long) * 8 * (size_t)cap));
  BP_CHECK(cudaMalloc(&h->d_vb2hi, sizeof(int64_t) * (size_t)cap));
  BP_CHECK(cudaMemset(h->d_isums, 0, sizeof(long long) * 8 * (size_t)cap));
  BP_CHECK(cudaMemset(h->d_keys, 0, sizeof(unsigned long long) * (size_t)cap));
  BP_CHECK(cudaMemset(h->d_done, 0, sizeof(unsigned int) * (size_t)cap));
  h->cap_batch = cap;
  return BP_OK;
}

EvalArgs blank_args() {
  EvalArgs A;
  std::memset(&A, 0, sizeof(A));
  A.one = 1u;
  return A;
}

// Dynamic shared memory of the prefix-count kernel.
size_t prefix_smem(int mode, int64_t max_bins) {
  return (size_t)kPrefixSmemBytes + (mode == kSrcNodes ? sizeof(uint32_t) * (size_t)max_bins : 0);
}

int launch_prefix(int mode, unsigned grid, size_t smem, cudaStream_t st, EvalArgs &A,
                  bool pdl = false) {
  return launch_fn((const void *)prefix_fn(mode), grid, kPrefixNT, smem, st, A, pdl);
}

// Dynamic shared memory of the cluster kernel: a table slice, the
// per-parameter accumulators, then (search nodes) the bin loads.
size_t cluster_smem(int mode, int64_t max_bins) {
  return (size_t)(kSliceBytes + kOwnBytes) +
         (mode == kSrcNodes ? sizeof(uint32_t) * (size_t)max_bins : 0);
}

// Clusters of the cluster kernel resident at once at `smem` bytes per CTA.
int cluster_slots(bp_lb *h, int mode, size_t smem) {
  if (h->cl_smem[mode] == smem && h->cl_clusters[mode] > 0) return h->cl_clusters[mode];
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(kClusterCtas * h->num_sms));
  cfg.blockDim = dim3(kPrefixNT);
  cfg.dynamicSmemBytes = smem;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void *)cluster_fn(mode), &cfg) != cudaSuccess)
    return 0;
  h->cl_smem[mode] = smem;
  h->cl_clusters[mode] = n;
  return n;
}

// The cluster kernel over `clusters` clusters (the grid is kClusterCtas times
// that; the kernel's cluster shape is compiled in).
int launch_cluster(int mode, unsigned clusters, size_t smem, cudaStream_t st, EvalArgs &A) {
  void *args[] = {&A};
  return cuda_status(cudaLaunchKernel((const void *)cluster_fn(mode),
                                      dim3(clusters * (unsigned)kClusterCtas), dim3(kPrefixNT),
                                      args, smem, st));
}

// The prefix_on bits for a call whose prefix kernel runs `ctas` CTAs: the
// global-table bit only when the scratch covers them (allocated on first use;
// if that fails, tables stay in shared memory).
int32_t prefix_bits(bp_lb *h, bool on, int64_t ctas) {
  if (!on) return 0;
  if (!h->d_gscratch && !h->gscratch_failed) {
    const int64_t n = (int64_t)h->num_sms * 4;  // the prefix kernel's most resident CTAs
    if (cudaMalloc(&h->d_gscratch, sizeof(int32_t) * (size_t)kGlobalTableInts * (size_t)n) ==
        cudaSuccess) {
      h->gscratch_ctas = n;
    } else {
      cudaGetLastError();  // clear the allocation error
      h->d_gscratch = nullptr;
      h->gscratch_failed = true;
    }
  }
  return kPrefixShared | ((h->d_gscratch && ctas <= h->gscratch_ctas) ? kPrefixGlobal : 0) |
         (h->cluster_on ? kPrefixCluster : 0);
}

// VB2's cap (vb2cap_kernel) of the A.B instances into hi[0 .. A.B).
int launch_vb2cap(bp_lb *h, int mode, const EvalArgs &A, int64_t *hi, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<int64_t>(A.B, (int64_t)h->num_sms * 8);
  const size_t smem = mode == kSrcNodes ? sizeof(uint32_t) * (size_t)A.max_bins : 0;
  if (mode == kSrcRaggedI32)
    vb2cap_kernel<256, kSrcRaggedI32><<<grid, 256, smem, st>>>(A, hi);
  else if (mode == kSrcRaggedI64)
    vb2cap_kernel<256, kSrcRaggedI64><<<grid, 256, smem, st>>>(A, hi);
  else
    vb2cap_kernel<256, kSrcNodes><<<grid, 256, smem, st>>>(A, hi);
  return cuda_status(cudaGetLastError());
}

// Dynamic shared memory of the VB2 kernel.
size_t vb2_smem(int mode, int64_t max_bins) {
  return kVb2ListBytes + (mode == kSrcNodes ? sizeof(uint32_t) * (size_t)max_bins : 0);
}

// Next event of the timing pool (grown on demand; timing is for measurement
// runs, not for stream capture).
cudaEvent_t next_event(bp_lb *h) {
  if (h->ev_next == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_next++];
}

template <int MODE>
int launch_batch(bp_lb *h, EvalArgs A, size_t smem, cudaStream_t st) {
  if (A.B == 0) return BP_OK;
  const int s = grow_batch(h, A.B);
  if (s != BP_OK) return s;
  A.tile_start = h->d_tile_start;
  A.keys = h->d_keys;
  A.done = h->d_done;
  A.work = h->d_work;
  A.prefix_on = prefix_bits(h, h->prefix_on != 0, (int64_t)h->num_sms * 4);
  A.gscratch = h->d_gscratch;
  A.ptile_start = h->d_ptile_start;
  A.pwork = h->d_work + 1;
  A.plpt = kPrefixLPTBatch;
  A.ctile_start = h->d_ctile_start;
  A.cwork = h->d_work + 4;
  A.vb2_on = h->vb2_on;
  A.verdict = h->verdict;
  A.prune = h->prune;
  A.reduce_mode = h->reduce_mode;
  A.dff_off = h->dff_off;
  A.work_count = h->timing ? h->d_work_count : nullptr;
  A.isums = h->d_isums;
  A.vtile_start = h->d_vtile_start;
  A.vwork = h->d_work + 2;
  A.vlpt = reinterpret_cast<long long *>(h->d_work + 3);
  A.vb2_target_tiles = (int64_t)h->num_sms * kVb2TilesPerSm;
  const int shape = h->shape[MODE];
  const int occ = occupancy(h, MODE, smem);
  if (occ <= 0) return BP_ECUDA;
  plan_kernel<MODE><<<1, 1024, 0, st>>>(A, shape_lpt(shape), h->d_tile_start, h->d_ptile_start,
                                        h->d_vtile_start, h->d_ctile_start);
  BP_CHECK(cudaGetLastError());
  if (h->vb2_cap) {
    // each instance's last VB2 parameter under the cap, before any VB2 tile
    A.vb2_hi = h->d_vb2hi;
    BP_CHECK_STATUS(launch_vb2cap(h, MODE, A, h->d_vb2hi, st));
  }
  // Timing events: [0] before the prefix kernel, [1] after it, [2] before the
  // VB2 kernel, [3] after it, [4] before the generic kernel, [5] after it,
  // [6] before the cluster kernel, [7] after it.
  std::array<cudaEvent_t, 8> ev = {nullptr, nullptr, nullptr, nullptr,
                                   nullptr, nullptr, nullptr, nullptr};
  if (h->timing)
    for (auto &e : ev)
      if (!(e = next_event(h))) return BP_ECUDA;
  const size_t ps = prefix_smem(MODE, A.max_bins);
  int pocc = 0;
  if (h->prefix_on) {
    BP_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pocc, (const void *)prefix_fn(MODE),
                                                           kPrefixNT, ps));
    if (pocc <= 0) return BP_ECUDA;
    pocc = std::min(pocc, 4);  // the global scratch covers num_sms x 4 CTAs
  }
  // With overlap, the prefix kernel (latency-bound table lookups) and then the
  // generic kernel run on the side stream while the VB2 kernel (bound by
  // integer issue) takes the rest of every SM; VB2's CTAs that do not fit at
  // first become resident as the prefix kernel's retire.  Stream-ordered
  // (fork after the plan, join before returning), so capturable in a graph.
  const bool overlap = h->prefix_ctas > 0 && h->vb2_on;
  cudaStream_t ps_st = overlap ? h->side : st;
  // The cluster kernel runs on the side stream, beside the prefix and VB2
  // kernels (where it finds no unit -- no instance with tables of its size --
  // its launch then costs the caller's stream nothing); the generic kernel
  // waits for it, since it publishes the instance sums that the generic
  // kernel's VB2 tiles are pruned with.  With overlap it simply leads the
  // side stream's sequence.
  const bool cl = (A.prefix_on & kPrefixCluster) != 0;
  const bool cl_side = cl && !overlap;
  if (overlap || cl_side) {
    BP_CHECK(cudaEventRecord(h->ev_fork, st));
    BP_CHECK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  }
  if (h->timing) BP_CHECK(cudaEventRecord(ev[6], h->side));
  if (cl) {
    const size_t cs = cluster_smem(MODE, A.max_bins);
    const int nc = cluster_slots(h, MODE, cs);
    if (nc <= 0) return BP_ECUDA;
    BP_CHECK_STATUS(launch_cluster(MODE, (unsigned)nc, cs, h->side, A));
  }
  if (h->timing) {
    if (cl) BP_CHECK(cudaEventRecord(ev[7], h->side));
    else ev[7] = ev[6];  // no cluster kernel: no time
  }
  if (cl_side) BP_CHECK(cudaEventRecord(h->ev_cjoin, h->side));
  // Serial order on the caller's stream with nothing between the kernels:
  // programmatic dependent launch (pdl_wait), so that each kernel is
  // scheduled while the one before it finishes.  Per-kernel timing events
  // sit between the kernels, so timed calls launch them plainly.
  const bool pdl = !overlap && !cl_side && !h->timing;
  if (h->timing) BP_CHECK(cudaEventRecord(ev[0], ps_st));
  if (h->prefix_on) {
    const int pc = overlap ? std::min(pocc, (int)h->prefix_ctas) : pocc;
    BP_CHECK_STATUS(launch_prefix(MODE, (unsigned)(h->num_sms * pc), ps, ps_st, A, pdl));
  }
  if (h->timing) BP_CHECK(cudaEventRecord(ev[1], ps_st));
  auto generic = [&](cudaStream_t gs) -> int {
    if (h->timing) BP_CHECK(cudaEventRecord(ev[4], gs));
    BP_CHECK_STATUS(launch_eval(shape, MODE, (unsigned)(h->num_sms * occ), smem, gs, A,
                                pdl && gs == st));
    if (h->timing) BP_CHECK(cudaEventRecord(ev[5], gs));
    return BP_OK;
  };
  if (overlap) {
    BP_CHECK_STATUS(generic(h->side));
    BP_CHECK(cudaEventRecord(h->ev_join, h->side));
  }
  if (h->timing) BP_CHECK(cudaEventRecord(ev[2], st));
  if (h->vb2_on) {
    // VB2's tiles on their own kernel (empty when no instance has any)
    const size_t vs = vb2_smem(MODE, A.max_bins);
    int vocc = 0;
    BP_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &vocc, (const void *)vb2_fn(shape, MODE), kVb2NT, vs));
    if (vocc <= 0) return BP_ECUDA;
    BP_CHECK_STATUS(launch_fn((const void *)vb2_fn(shape, MODE), (unsigned)(h->num_sms * vocc),
                              kVb2NT, vs, st, A, pdl));
  }
  if (h->timing) BP_CHECK(cudaEventRecord(ev[3], st));
  if (overlap) {
    BP_CHECK(cudaStreamWaitEvent(st, h->ev_join, 0));
  } else {
    if (cl_side) BP_CHECK(cudaStreamWaitEvent(st, h->ev_cjoin, 0));
    BP_CHECK_STATUS(generic(st));
  }
  if (h->timing) h->ev_pending.push_back(ev);
  return BP_OK;
}

// Times `reps` calls of `call` per launch shape with CUDA events on `st`,
// leaves the fastest shape set for `mode`.
template <class F>
int autotune(bp_lb *h, int mode, int32_t B, int32_t reps, cudaStream_t st, float *ms_out,
             int32_t *best_out, F call) {
  if (reps < 1) return BP_EINVAL;
  cudaEvent_t e0, e1;
  BP_CHECK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BP_ECUDA;
  }
  int best = 0, st_all = BP_OK;
  float best_ms = 0.f;
  for (int s = 0; s < kNumShapes && st_all == BP_OK; ++s) {
    h->shape[mode] = s;
    st_all = call();  // warm-up (also sets up occupancy)
    if (st_all != BP_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && st_all == BP_OK; ++r) st_all = call();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) st_all = BP_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms_out) ms_out[s] = ms;
    if (s == 0 || ms < best_ms) {
      best_ms = ms;
      best = s;
    }
  }
  h->shape[mode] = best;
  // then, with that shape, cluster tables switched: the faster setting stays
  // (on only when the batch has units for the cluster kernel: the planner's
  // count of them, read back after a call with them on)
  if (st_all == BP_OK) {
    const int32_t keep = h->cluster_on;
    h->cluster_on = !keep;
    st_all = call();
    float ms = 0.f;
    bool no_units = false;
    if (st_all == BP_OK && h->cluster_on) {
      int64_t units = 0;
      if (cudaMemcpyAsync(&units, h->d_ctile_start + B, sizeof(int64_t), cudaMemcpyDeviceToHost,
                          st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        st_all = BP_ECUDA;
      no_units = units == 0;
    }
    if (st_all == BP_OK && !no_units) {
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && st_all == BP_OK; ++r) st_all = call();
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) st_all = BP_ECUDA;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
    }
    // switched only for a clear gain (the setting costs a launch when it
    // finds nothing to do, and ties are noise)
    if (st_all != BP_OK || no_units || ms > 0.97f * best_ms) h->cluster_on = keep;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_out) *best_out = best;
  return st_all;
}

}  // namespace

extern "C" {

const char *bp_lb_strerror(int status) {
  switch (status) {
    case BP_OK: return "ok";
    case BP_EINVAL: return "invalid argument";
    case BP_ERANGE: return "value out of range";
    case BP_ENOMEM: return "out of memory";
    case BP_ECUDA: return "CUDA error";
    case BP_ETIMEOUT: return "timed out";
    case BP_EBUSY: return "busy: admission refused";
    default: return "unknown status";
  }
}

int bp_lb_create(int64_t capacity, int64_t max_items, bp_lb_t **out) {
  if (!out) return BP_EINVAL;
  *out = nullptr;
  if (capacity < 1 || capacity > kMaxCapacity || max_items < 1 || max_items > kMaxItems)
    return BP_ERANGE;
  bp_lb *h = new (std::nothrow) bp_lb();
  if (!h) return BP_ENOMEM;
  h->capacity = capacity;
  h->max_items = max_items;
  int st = BP_OK;
  do {
    if ((st = cuda_status(cudaGetDevice(&h->device))) != BP_OK) break;
    if ((st = cuda_status(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount,
                                                 h->device))) != BP_OK)
      break;
    if ((st = cuda_status(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking))) != BP_OK)
      break;
    int prio_lo = 0, prio_hi = 0;
    if ((st = cuda_status(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi))) != BP_OK) break;
    if ((st = cuda_status(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_hi))) !=
        BP_OK)
      break;
    if ((st = cuda_status(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming))) != BP_OK)
      break;
    if ((st = cuda_status(cudaEventCreateWithFlags(&h->ev_cjoin, cudaEventDisableTiming))) !=
        BP_OK)
      break;
    if ((st = cuda_status(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming))) != BP_OK)
      break;
    const size_t nb = sizeof(int32_t) * (size_t)max_items;
    if ((st = cuda_status(cudaMalloc(&h->d_items, nb))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_assign, nb))) != BP_OK) break;
    if ((st = cuda_status(cudaMallocHost(&h->h_items, nb))) != BP_OK) break;
    if ((st = cuda_status(cudaMallocHost(&h->h_assign, nb))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_out, sizeof(PlainOut)))) != BP_OK) break;
    if ((st = cuda_status(cudaMallocHost(&h->h_out, sizeof(PlainOut)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_key1, sizeof(unsigned long long)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_done1, sizeof(unsigned int)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_work, 8 * sizeof(unsigned long long)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_vb2hi1, sizeof(int64_t)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_rkey, sizeof(unsigned long long)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_rdone, sizeof(unsigned int)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_rout, sizeof(PlainOut)))) != BP_OK) break;
    if ((st = cuda_status(cudaMalloc(&h->d_rvb2hi, sizeof(int64_t)))) != BP_OK) break;
    if ((st = cuda_status(cudaMemset(h->d_rkey, 0, sizeof(unsigned long long)))) != BP_OK) break;
    if ((st = cuda_status(cudaMemset(h->d_rdone, 0, sizeof(unsigned int)))) != BP_OK) break;
    if ((st = cuda_status(cudaMemset(h->d_key1, 0, sizeof(unsigned long long)))) != BP_OK) break;
    if ((st = cuda_status(cudaMemset(h->d_done1, 0, sizeof(unsigned int)))) != BP_OK) break;
    if ((st = cuda_status(cudaMemset(h->d_work, 0, 8 * sizeof(unsigned long long)))) != BP_OK)
      break;
    for (int mode = 0; mode < 3 && st == BP_OK; ++mode) {
      st = cuda_status(cudaFuncSetAttribute((const void *)prefix_fn(mode),
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)prefix_smem(mode, kMaxNodeBins)));
      if (st == BP_OK)
        st = cuda_status(cudaFuncSetAttribute((const void *)cluster_fn(mode),
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)cluster_smem(mode, kMaxNodeBins)));
    }
    if (st != BP_OK) break;
    // the plain node path may use the full on-chip bin table
    const size_t smem_nodes = eval_smem<kSrcNodes>(kMaxNodeBins);
    for (int sh = 0; sh < kNumShapes && st == BP_OK; ++sh) {
      st = cuda_status(cudaFuncSetAttribute((const void *)eval_fn(sh, kSrcNodes),
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_nodes));
      if (st == BP_OK)
        st = cuda_status(cudaFuncSetAttribute((const void *)vb2_fn(sh, kSrcNodes),
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)vb2_smem(kSrcNodes, kMaxNodeBins)));
    }
    if (st != BP_OK) break;
    if ((st = cuda_status(cudaFuncSetAttribute(l2_kernel<kL2NT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kL2SmemBytes))) != BP_OK)
      break;
    if ((st = cuda_status(cudaFuncSetAttribute(vb2cap_kernel<256, kSrcNodes>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(uint32_t) * kMaxNodeBins)))) != BP_OK)
      break;
    if ((st = cuda_status(cudaFuncSetAttribute(reduce_kernel<256>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)(sizeof(uint32_t) * kMaxNodeBins)))) != BP_OK)
      break;
    if ((st = cuda_status(cudaDeviceSynchronize())) != BP_OK) break;
  } while (0);
  if (st != BP_OK) {
    bp_lb_destroy(h);
    return st;
  }
  *out = h;
  return BP_OK;
}

int bp_lb_destroy(bp_lb_t *h) {
  if (!h) return BP_OK;
  cudaDeviceSynchronize();
  cudaFree(h->d_items);
  cudaFree(h->d_assign);
  cudaFreeHost(h->h_items);
  cudaFreeHost(h->h_assign);
  cudaFree(h->d_out);
  cudaFreeHost(h->h_out);
  cudaFree(h->d_key1);
  cudaFree(h->d_done1);
  cudaFree(h->d_work);
  cudaFree(h->d_tile_start);
  cudaFree(h->d_ptile_start);
  cudaFree(h->d_vtile_start);
  cudaFree(h->d_keys);
  cudaFree(h->d_done);
  cudaFree(h->d_gscratch);
  cudaFree(h->d_work_count);
  cudaFree(h->d_isums);
  cudaFree(h->d_vb2hi);
  cudaFree(h->d_vb2hi1);
  cudaFree(h->d_rkey);
  cudaFree(h->d_rdone);
  cudaFree(h->d_rout);
  cudaFree(h->d_rvb2hi);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_cjoin) cudaEventDestroy(h->ev_cjoin);
  delete h;
  return BP_OK;
}

int bp_lb_reserve(bp_lb_t *h, int32_t max_batch) {
  if (!h || max_batch < 0) return BP_EINVAL;
  return grow_batch(h, max_batch);
}

static int plain_finish(bp_lb *h, int64_t *out_bound, bp_argmax_t *out_argmax) {
  BP_CHECK(cudaMemcpyAsync(h->h_out, h->d_out, sizeof(PlainOut), cudaMemcpyDeviceToHost, h->stream));
  BP_CHECK(cudaStreamSynchronize(h->stream));
  if (h->h_out->bound < 0) return BP_ERANGE;
  *out_bound = h->h_out->bound;
  if (out_argmax) *out_argmax = h->h_out->arg;
  return BP_OK;
}

// The plain result when no parameter is left to evaluate (every DFF left in
// has an empty range at this capacity): bound 0, no argmax.
static int plain_empty(int64_t *out_bound, bp_argmax_t *out_argmax) {
  *out_bound = 0;
  if (out_argmax) {
    out_argmax->dff = -1;
    out_argmax->pad = 0;
    out_argmax->lambda = -1;
  }
  return BP_OK;
}

static EvalArgs plain_args(bp_lb *h, int64_t n, int64_t bins, int mode) {
  EvalArgs A = blank_args();
  A.B = 1;
  A.out_bound = &h->d_out->bound;
  A.out_argmax = &h->d_out->arg;
  A.out_feasible = &h->d_out->feasible;
  A.tile_start = nullptr;
  // mode is a plain mode; the sum bound is the stream length times c
  const int64_t sb = (mode == kModePlainNodes ? n + bins : n) * h->capacity;
  A.vb2_on = 0;
  A.verdict = h->verdict;
  A.prune = h->prune;
  A.reduce_mode = h->reduce_mode;
  A.dff_off = h->dff_off;
  A.plpt = kPrefixLPTSingle;
  // global prefix tables when the scratch covers the prefix tiles (one CTA each)
  A.prefix_on = prefix_bits(h, h->plain_prefix_on != 0, 0);
  if (A.prefix_on & kPrefixGlobal) {
    const int64_t pt = route_tiles(kRoutePrefix, h->capacity, A.plpt, sb, A.prefix_on, 0, A.dff_off);
    if (pt > h->gscratch_ctas) A.prefix_on &= ~kPrefixGlobal;
  }
  A.gscratch = h->d_gscratch;
  A.single_tiles = route_tiles(kRouteDirect, h->capacity, shape_lpt(h->shape[mode]), sb,
                               A.prefix_on, 0, A.dff_off);
  A.single_ptiles = route_tiles(kRoutePrefix, h->capacity, A.plpt, sb, A.prefix_on, 0, A.dff_off);
  A.single_ctiles = route_tiles(kRouteCluster, h->capacity, A.plpt, sb, A.prefix_on, 0, A.dff_off);
  A.single_vtiles = 0;
  A.single_c = h->capacity;
  A.single_k = bins;
  A.single_n = n;
  A.keys = h->d_key1;
  A.done = h->d_done1;
  A.work = nullptr;
  return A;
}

int bp_lb_eval(bp_lb_t *h, const int32_t *sizes, int64_t n, int64_t bins, int64_t *out_bound,
               bp_argmax_t *out_argmax) {
  if (!h || !out_bound || (n > 0 && !sizes) || n < 0 || bins < 0) return BP_EINVAL;
  if (n > h->max_items) return BP_ERANGE;
  const int64_t c = h->capacity;
  for (int64_t i = 0; i < n; ++i)
    if (sizes[i] < 0 || (int64_t)sizes[i] > c) return BP_ERANGE;
  if (n > 0) {
    std::memcpy(h->h_items, sizes, sizeof(int32_t) * (size_t)n);
    BP_CHECK(cudaMemcpyAsync(h->d_items, h->h_items, sizeof(int32_t) * (size_t)n,
                             cudaMemcpyHostToDevice, h->stream));
  }
  EvalArgs A = plain_args(h, n, bins, kModePlainRagged);
  A.sizes = h->d_items;
  if (A.single_ptiles + A.single_tiles + A.single_ctiles == 0)
    return plain_empty(out_bound, out_argmax);
  if (h->vb2_cap) {
    A.vb2_hi = h->d_vb2hi1;
    BP_CHECK_STATUS(launch_vb2cap(h, kSrcRaggedI32, A, h->d_vb2hi1, h->stream));
  }
  if (A.single_ctiles > 0)
    BP_CHECK_STATUS(launch_cluster(kSrcRaggedI32, (unsigned)A.single_ctiles,
                                   cluster_smem(kSrcRaggedI32, 0), h->stream, A));
  if (A.single_ptiles > 0)
    BP_CHECK_STATUS(launch_prefix(kSrcRaggedI32, (unsigned)A.single_ptiles,
                                  prefix_smem(kSrcRaggedI32, 0), h->stream, A));
  if (A.single_tiles > 0)
    BP_CHECK_STATUS(launch_eval(h->shape[kModePlainRagged], kSrcRaggedI32,
                                (unsigned)A.single_tiles, eval_smem<kSrcRaggedI32>(0), h->stream, A));
  return plain_finish(h, out_bound, out_argmax);
}

int bp_lb_eval_node(bp_lb_t *h, const int32_t *w, const int32_t *assign, int64_t n, int64_t bins,
                    int64_t *out_bound, bp_argmax_t *out_argmax) {
  if (!h || !out_bound || (n > 0 && (!w || !assign)) || n < 0 || bins < 0) return BP_EINVAL;
  if (n > h->max_items || bins > h->max_items || bins > kMaxNodeBins) return BP_ERANGE;
  if (n > 0) {
    std::memcpy(h->h_items, w, sizeof(int32_t) * (size_t)n);
    std::memcpy(h->h_assign, assign, sizeof(int32_t) * (size_t)n);
    BP_CHECK(cudaMemcpyAsync(h->d_items, h->h_items, sizeof(int32_t) * (size_t)n,
                             cudaMemcpyHostToDevice, h->stream));
    BP_CHECK(cudaMemcpyAsync(h->d_assign, h->h_assign, sizeof(int32_t) * (size_t)n,
                             cudaMemcpyHostToDevice, h->stream));
  }
  EvalArgs A = plain_args(h, n, bins, kModePlainNodes);
  A.base_sizes = h->d_items;
  A.assign = h->d_assign;
  A.max_bins = (int32_t)bins;
  if (A.single_ptiles + A.single_tiles + A.single_ctiles == 0)
    return plain_empty(out_bound, out_argmax);
  if (h->vb2_cap) {
    A.vb2_hi = h->d_vb2hi1;
    BP_CHECK_STATUS(launch_vb2cap(h, kSrcNodes, A, h->d_vb2hi1, h->stream));
  }
  if (A.single_ctiles > 0)
    BP_CHECK_STATUS(launch_cluster(kSrcNodes, (unsigned)A.single_ctiles,
                                   cluster_smem(kSrcNodes, bins), h->stream, A));
  if (A.single_ptiles > 0)
    BP_CHECK_STATUS(launch_prefix(kSrcNodes, (unsigned)A.single_ptiles, prefix_smem(kSrcNodes, bins),
                                  h->stream, A));
  if (A.single_tiles > 0)
    BP_CHECK_STATUS(launch_eval(h->shape[kModePlainNodes], kSrcNodes, (unsigned)A.single_tiles,
                                eval_smem<kSrcNodes>(bins), h->stream, A));
  return plain_finish(h, out_bound, out_argmax);
}

int bp_lb_eval_batch(bp_lb_t *h, int32_t B, const int64_t *d_offsets, const int32_t *d_sizes,
                     const int64_t *d_capacity, const int64_t *d_bins, int64_t *d_out_bound,
                     bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible, void *stream) {
  if (!h || B < 0) return BP_EINVAL;
  if (B == 0) return BP_OK;
  if (!d_offsets || !d_sizes || !d_capacity || !d_bins || !d_out_bound) return BP_EINVAL;
  EvalArgs A = blank_args();
  A.B = B;
  A.offsets = d_offsets;
  A.sizes = d_sizes;
  A.capacity = d_capacity;
  A.bins = d_bins;
  A.out_bound = d_out_bound;
  A.out_argmax = d_out_argmax;
  A.out_feasible = d_out_feasible;
  return launch_batch<kSrcRaggedI32>(h, A, eval_smem<kSrcRaggedI32>(0), (cudaStream_t)stream);
}

int bp_lb_eval_batch_i64(bp_lb_t *h, int32_t B, const int64_t *d_offsets, const int64_t *d_sizes,
                         const int64_t *d_capacity, const int64_t *d_bins, int64_t *d_out_bound,
                         bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible, void *stream) {
  if (!h || B < 0) return BP_EINVAL;
  if (B == 0) return BP_OK;
  if (!d_offsets || !d_sizes || !d_capacity || !d_bins || !d_out_bound) return BP_EINVAL;
  EvalArgs A = blank_args();
  A.B = B;
  A.offsets = d_offsets;
  A.sizes = d_sizes;
  A.capacity = d_capacity;
  A.bins = d_bins;
  A.out_bound = d_out_bound;
  A.out_argmax = d_out_argmax;
  A.out_feasible = d_out_feasible;
  return launch_batch<kSrcRaggedI64>(h, A, eval_smem<kSrcRaggedI64>(0), (cudaStream_t)stream);
}

int bp_lb_eval_nodes(bp_lb_t *h, int32_t B, int32_t num_base, const int64_t *d_base_offsets,
                     const int32_t *d_base_sizes, const int64_t *d_base_capacity,
                     const int32_t *d_node_base, const int64_t *d_assign_offsets,
                     const int32_t *d_assign, const int64_t *d_bins, int64_t max_bins,
                     int64_t *d_out_bound, bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                     void *stream) {
  if (!h || B < 0 || num_base < 0) return BP_EINVAL;
  if (max_bins < 0 || max_bins > kMaxNodeBins) return BP_ERANGE;
  if (B == 0) return BP_OK;
  if (!d_base_offsets || !d_base_sizes || !d_base_capacity || !d_node_base || !d_assign_offsets ||
      !d_assign || !d_bins || !d_out_bound)
    return BP_EINVAL;
  EvalArgs A = blank_args();
  A.B = B;
  A.num_base = num_base;
  A.base_offsets = d_base_offsets;
  A.base_sizes = d_base_sizes;
  A.base_capacity = d_base_capacity;
  A.node_base = d_node_base;
  A.assign_offsets = d_assign_offsets;
  A.assign = d_assign;
  A.bins = d_bins;
  A.max_bins = (int32_t)max_bins;
  A.out_bound = d_out_bound;
  A.out_argmax = d_out_argmax;
  A.out_feasible = d_out_feasible;
  A.bin_max_offsets = h->d_bin_max_offsets;
  A.bin_max = h->d_bin_max;
  return launch_batch<kSrcNodes>(h, A, eval_smem<kSrcNodes>(max_bins), (cudaStream_t)stream);
}

int bp_lb_reduce_nodes(bp_lb_t *h, int32_t B, int32_t num_base, const int64_t *d_base_offsets,
                       const int32_t *d_base_sizes, const int64_t *d_base_capacity,
                       const int32_t *d_node_base, const int64_t *d_assign_offsets,
                       const int32_t *d_assign, const int64_t *d_bins, int64_t max_bins,
                       const int64_t *d_out_offsets, int32_t *d_out_sizes, int64_t *d_out_count,
                       void *stream) {
  if (!h || B < 0 || num_base < 0) return BP_EINVAL;
  if (max_bins < 0 || max_bins > kMaxNodeBins) return BP_ERANGE;
  if (B == 0) return BP_OK;
  if (!d_base_offsets || !d_base_sizes || !d_base_capacity || !d_node_base || !d_assign_offsets ||
      !d_assign || !d_bins || !d_out_offsets || !d_out_sizes || !d_out_count)
    return BP_EINVAL;
  EvalArgs A = blank_args();
  A.B = B;
  A.num_base = num_base;
  A.base_offsets = d_base_offsets;
  A.base_sizes = d_base_sizes;
  A.base_capacity = d_base_capacity;
  A.node_base = d_node_base;
  A.assign_offsets = d_assign_offsets;
  A.assign = d_assign;
  A.bins = d_bins;
  A.max_bins = (int32_t)max_bins;
  A.reduce_mode = h->reduce_mode;
  A.bin_max_offsets = h->d_bin_max_offsets;
  A.bin_max = h->d_bin_max;
  const int grid = (int)std::min<int64_t>(B, (int64_t)h->num_sms * 8);
  reduce_kernel<256><<<grid, 256, sizeof(uint32_t) * (size_t)max_bins, (cudaStream_t)stream>>>(
      A, d_out_offsets, d_out_sizes, d_out_count);
  BP_CHECK(cudaGetLastError());
  return BP_OK;
}

int bp_lb_l2_batch(bp_lb_t *h, int32_t B, const int64_t *d_offsets, const int32_t *d_sizes,
                   const int64_t *d_capacity, int64_t *d_out_l2, void *stream) {
  if (!h || B < 0) return BP_EINVAL;
  if (B == 0) return BP_OK;
  if (!d_offsets || !d_sizes || !d_capacity || !d_out_l2) return BP_EINVAL;
  const int grid = (int)std::min<int64_t>(B, (int64_t)h->num_sms * 2);
  l2_kernel<kL2NT><<<grid, kL2NT, kL2SmemBytes, (cudaStream_t)stream>>>(B, d_offsets, d_sizes,
                                                                       d_capacity, d_out_l2);
  BP_CHECK(cudaGetLastError());
  return BP_OK;
}

int bp_lb_debug_params(bp_lb_t *h, const int32_t *d_sizes, int64_t n, int64_t c,
                       const int32_t *d_dff, const int64_t *d_lambda, int64_t m, int64_t *d_out_lb,
                       void *stream) {
  if (!h || n < 0 || m < 0 || (n > 0 && !d_sizes)) return BP_EINVAL;
  if (c < 1 || c > kMaxCapacity || n > kMaxItems) return BP_ERANGE;
  if (m == 0) return BP_OK;
  if (!d_dff || !d_lambda || !d_out_lb) return BP_EINVAL;
  EvalArgs A = blank_args();
  A.B = 1;
  A.sizes = d_sizes;
  A.single_c = c;
  A.single_k = 0;
  A.single_n = n;
  A.single_tiles = 1;
  const dim3 grid((unsigned)((m + 255) / 256), kNumDff);
  debug_kernel<256><<<grid, 256, kListBytes, (cudaStream_t)stream>>>(A, d_dff, d_lambda, m,
                                                                     d_out_lb);
  BP_CHECK(cudaGetLastError());
  return BP_OK;
}

int bp_lb_eval_range(bp_lb_t *h, const int32_t *d_sizes, int64_t n, int64_t c, int64_t g0,
                     int64_t g1, int64_t *d_out_key, void *stream) {
  if (!h || n < 0 || (n > 0 && !d_sizes) || !d_out_key) return BP_EINVAL;
  if (c < 1 || c > kMaxCapacity || n > kMaxItems) return BP_ERANGE;
  if (g0 < 0 || g0 > g1 || g1 > param_total(c)) return BP_ERANGE;
  cudaStream_t st = (cudaStream_t)stream;
  EvalArgs A = blank_args();
  A.B = 1;
  A.sizes = d_sizes;
  A.single_c = c;
  A.single_k = 0;
  A.single_n = n;
  A.out_bound = &h->d_rout->bound;
  A.out_argmax = &h->d_rout->arg;
  A.out_feasible = &h->d_rout->feasible;
  A.out_key = d_out_key;
  A.windowed = 1;
  A.g_lo = (uint32_t)g0;
  A.g_hi = (uint32_t)g1;
  A.prefix_on = 0;  // every parameter item by item in the generic kernel
  A.vb2_on = 0;
  A.prune = h->prune;  // VB2 against this window's own best key so far (exact)
  A.dff_off = h->dff_off;
  A.keys = h->d_rkey;
  A.done = h->d_rdone;
  const int shape = h->shape[BP_MODE_RAGGED_I32];
  const int64_t lpt = shape_lpt(shape);
  int64_t tiles = 0;
  for (int d = 0; d < kNumDff; ++d) {
    if ((h->dff_off >> d) & 1u) continue;
    int64_t lo, hi;
    tiles += (window_range(d, c, 1, (uint32_t)g0, (uint32_t)g1, lo, hi) + lpt - 1) / lpt;
  }
  A.single_tiles = tiles;
  if (tiles == 0) {  // no parameter in the window: key 0
    BP_CHECK(cudaMemsetAsync(d_out_key, 0, sizeof(int64_t), st));
    return BP_OK;
  }
  if (h->vb2_cap) {
    A.vb2_hi = h->d_rvb2hi;
    BP_CHECK_STATUS(launch_vb2cap(h, kSrcRaggedI32, A, h->d_rvb2hi, st));
  }
  return launch_eval(shape, kSrcRaggedI32, (unsigned)tiles, eval_smem<kSrcRaggedI32>(0), st, A);
}

int bp_lb_set_algorithm(bp_lb_t *h, int32_t algo) {
  if (!h) return BP_EINVAL;
  if (algo != BP_ALGO_DIRECT && algo != BP_ALGO_PREFIX) return BP_ERANGE;
  h->prefix_on = h->plain_prefix_on = algo == BP_ALGO_PREFIX;
  return BP_OK;
}

int bp_lb_set_vb2_cap(bp_lb_t *h, int32_t on) {
  if (!h) return BP_EINVAL;
  if (on != 0 && on != 1) return BP_ERANGE;
  h->vb2_cap = on;
  return BP_OK;
}

int bp_lb_get_vb2_cap(bp_lb_t *h) {
  if (!h) return -1;
  return h->vb2_cap;
}

int bp_lb_set_result_mode(bp_lb_t *h, int32_t mode) {
  if (!h) return BP_EINVAL;
  if (mode != BP_RESULT_FULL && mode != BP_RESULT_VERDICT) return BP_ERANGE;
  h->verdict = mode == BP_RESULT_VERDICT;
  return BP_OK;
}

int bp_lb_get_result_mode(bp_lb_t *h) {
  if (!h) return -1;
  return h->verdict ? BP_RESULT_VERDICT : BP_RESULT_FULL;
}

int bp_lb_set_reduction(bp_lb_t *h, int32_t mode) {
  if (!h) return BP_EINVAL;
  if (mode != BP_REDUCE_LOADS && mode != BP_REDUCE_CLOSE) return BP_ERANGE;
  h->reduce_mode = mode;
  return BP_OK;
}

int bp_lb_get_reduction(bp_lb_t *h) {
  if (!h) return -1;
  return h->reduce_mode;
}

int bp_lb_set_bin_max(bp_lb_t *h, const int64_t *d_offsets, const int32_t *d_bin_max) {
  if (!h) return BP_EINVAL;
  if ((d_offsets == nullptr) != (d_bin_max == nullptr)) return BP_EINVAL;
  h->d_bin_max_offsets = d_offsets;
  h->d_bin_max = d_bin_max;
  return BP_OK;
}

int bp_lb_set_pruning(bp_lb_t *h, int32_t on) {
  if (!h) return BP_EINVAL;
  if (on != 0 && on != 1) return BP_ERANGE;
  h->prune = on;
  return BP_OK;
}

int bp_lb_get_pruning(bp_lb_t *h) {
  if (!h) return -1;
  return h->prune;
}

int bp_lb_set_cluster_tables(bp_lb_t *h, int32_t on) {
  if (!h) return BP_EINVAL;
  if (on != 0 && on != 1) return BP_ERANGE;
  h->cluster_on = on;
  return BP_OK;
}

int bp_lb_get_cluster_tables(bp_lb_t *h) { return h ? h->cluster_on : -1; }

int bp_lb_set_overlap(bp_lb_t *h, int32_t prefix_ctas_per_sm) {
  if (!h) return BP_EINVAL;
  if (prefix_ctas_per_sm < 0 || prefix_ctas_per_sm > 8) return BP_ERANGE;
  h->prefix_ctas = prefix_ctas_per_sm;
  return BP_OK;
}

int bp_lb_set_dff_mask(bp_lb_t *h, int32_t mask) {
  if (!h) return BP_EINVAL;
  if (mask < 1 || mask > 63) return BP_ERANGE;
  h->dff_off = (~(uint32_t)mask) & 63u;
  return BP_OK;
}

int bp_lb_get_dff_mask(bp_lb_t *h) {
  if (!h) return -1;
  return (int)((~h->dff_off) & 63u);
}

int bp_lb_set_kernel_timing(bp_lb_t *h, int32_t on) {
  if (!h) return BP_EINVAL;
  if (on && !h->d_work_count) {
    BP_CHECK(cudaMalloc(&h->d_work_count, 4 * sizeof(unsigned long long)));
    BP_CHECK(cudaMemsetAsync(h->d_work_count, 0, 4 * sizeof(unsigned long long), h->stream));
    BP_CHECK(cudaStreamSynchronize(h->stream));
  }
  h->timing = on != 0;
  return BP_OK;
}

int bp_lb_kernel_work(bp_lb_t *h, int64_t *out4) {
  if (!h || !out4) return BP_EINVAL;
  unsigned long long v[4] = {0ull, 0ull, 0ull, 0ull};
  if (h->d_work_count) {
    BP_CHECK(cudaDeviceSynchronize());
    BP_CHECK(cudaMemcpy(v, h->d_work_count, sizeof(v), cudaMemcpyDeviceToHost));
    BP_CHECK(cudaMemset(h->d_work_count, 0, sizeof(v)));
  }
  for (int i = 0; i < 4; ++i) out4[i] = (int64_t)v[i];
  return BP_OK;
}

int bp_lb_kernel_times4(bp_lb_t *h, double *out_ms4, int64_t *calls) {
  if (!h) return BP_EINVAL;
  double p = 0.0, v = 0.0, d = 0.0, cl = 0.0;
  for (const auto &ev : h->ev_pending) {
    BP_CHECK(cudaEventSynchronize(ev[3]));
    BP_CHECK(cudaEventSynchronize(ev[5]));
    float a = 0.f, b = 0.f, e = 0.f, f = 0.f;
    BP_CHECK(cudaEventElapsedTime(&a, ev[0], ev[1]));
    BP_CHECK(cudaEventElapsedTime(&b, ev[2], ev[3]));
    BP_CHECK(cudaEventElapsedTime(&e, ev[4], ev[5]));
    BP_CHECK(cudaEventElapsedTime(&f, ev[6], ev[7]));
    p += a;
    v += b;
    d += e;
    cl += f;
  }
  if (out_ms4) {
    out_ms4[0] = cl;
    out_ms4[1] = p;
    out_ms4[2] = v;
    out_ms4[3] = d;
  }
  if (calls) *calls = (int64_t)h->ev_pending.size();
  h->ev_pending.clear();
  h->ev_next = 0;
  return BP_OK;
}

int bp_lb_kernel_times(bp_lb_t *h, double *ms_prefix, double *ms_vb2, double *ms_direct,
                       int64_t *calls) {
  double ms[4];
  const int st = bp_lb_kernel_times4(h, ms, calls);
  if (st != BP_OK) return st;
  if (ms_prefix) *ms_prefix = ms[1];
  if (ms_vb2) *ms_vb2 = ms[2];
  if (ms_direct) *ms_direct = ms[3];
  return BP_OK;
}

int bp_lb_get_algorithm(bp_lb_t *h) {
  if (!h) return -1;
  return h->prefix_on ? BP_ALGO_PREFIX : BP_ALGO_DIRECT;
}

int bp_lb_num_launch_shapes(void) { return kNumShapes; }

int bp_lb_launch_shape_info(int32_t id, int32_t *nt, int32_t *t, int32_t *g, int32_t *min_blocks) {
  if (id < 0 || id >= kNumShapes) return BP_ERANGE;
  if (nt) *nt = kShapes[id].nt;
  if (t) *t = kShapes[id].t;
  if (g) *g = kShapes[id].g;
  if (min_blocks) *min_blocks = kShapes[id].minb;
  return BP_OK;
}

int bp_lb_set_launch_shape(bp_lb_t *h, int32_t mode, int32_t id) {
  if (!h || mode < 0 || mode > 4) return BP_EINVAL;
  if (id < 0 || id >= kNumShapes) return BP_ERANGE;
  h->shape[mode] = id;
  return BP_OK;
}

int bp_lb_get_launch_shape(bp_lb_t *h, int32_t mode) {
  if (!h || mode < 0 || mode > 4) return -1;
  return h->shape[mode];
}

int bp_lb_autotune_plain_node(bp_lb_t *h, const int32_t *w, const int32_t *assign, int64_t n,
                              int64_t bins, int32_t reps, float *us_per_shape,
                              int32_t *best_shape) {
  if (!h || reps < 1) return BP_EINVAL;
  int best = h->shape[kModePlainNodes], best_algo = h->plain_prefix_on;
  double best_us = -1.0;
  for (int algo = 0; algo < 2; ++algo) {
    h->plain_prefix_on = algo;
    for (int s = 0; s < kNumShapes; ++s) {
      h->shape[kModePlainNodes] = s;
      int64_t b;
      int st = bp_lb_eval_node(h, w, assign, n, bins, &b, nullptr);  // warm-up
      if (st != BP_OK && st != BP_ERANGE) {
        h->shape[kModePlainNodes] = best;
        h->plain_prefix_on = best_algo;
        return st;
      }
      const auto t0 = std::chrono::steady_clock::now();
      for (int r = 0; r < reps; ++r) bp_lb_eval_node(h, w, assign, n, bins, &b, nullptr);
      const double us = std::chrono::duration<double, std::micro>(
                            std::chrono::steady_clock::now() - t0).count() / reps;
      if (us_per_shape) us_per_shape[algo * kNumShapes + s] = (float)us;
      if (best_us < 0 || us < best_us) {
        best_us = us;
        best = s;
        best_algo = algo;
      }
    }
  }
  h->shape[kModePlainNodes] = best;
  h->plain_prefix_on = best_algo;
  if (best_shape) *best_shape = best_algo * kNumShapes + best;
  return BP_OK;
}

int bp_lb_autotune_batch(bp_lb_t *h, int32_t B, const int64_t *d_offsets, const void *d_sizes,
                         int32_t sizes_are_i64, const int64_t *d_capacity, const int64_t *d_bins,
                         int64_t *d_out_bound, bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                         int32_t reps, float *ms_per_shape, int32_t *best_shape, void *stream) {
  if (!h || B < 1) return BP_EINVAL;
  const int mode = sizes_are_i64 ? kSrcRaggedI64 : kSrcRaggedI32;
  return autotune(h, mode, B, reps, (cudaStream_t)stream, ms_per_shape, best_shape, [&]() {
    return sizes_are_i64
               ? bp_lb_eval_batch_i64(h, B, d_offsets, (const int64_t *)d_sizes, d_capacity, d_bins,
                                      d_out_bound, d_out_argmax, d_out_feasible, stream)
               : bp_lb_eval_batch(h, B, d_offsets, (const int32_t *)d_sizes, d_capacity, d_bins,
                                  d_out_bound, d_out_argmax, d_out_feasible, stream);
  });
}

int bp_lb_autotune_nodes(bp_lb_t *h, int32_t B, int32_t num_base, const int64_t *d_base_offsets,
                         const int32_t *d_base_sizes, const int64_t *d_base_capacity,
                         const int32_t *d_node_base, const int64_t *d_assign_offsets,
                         const int32_t *d_assign, const int64_t *d_bins, int64_t max_bins,
                         int64_t *d_out_bound, bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                         int32_t reps, float *ms_per_shape, int32_t *best_shape, void *stream) {
  if (!h || B < 1) return BP_EINVAL;
  return autotune(h, kSrcNodes, B, reps, (cudaStream_t)stream, ms_per_shape, best_shape, [&]() {
    return bp_lb_eval_nodes(h, B, num_base, d_base_offsets, d_base_sizes, d_base_capacity,
                            d_node_base, d_assign_offsets, d_assign, d_bins, max_bins, d_out_bound,
                            d_out_argmax, d_out_feasible, stream);
  });
}

int bp_lb_dff_route(int32_t d, int64_t c, int64_t stream_len, int32_t algo) {
  if (d < 0 || d >= kNumDff || c < 1 || c > kMaxCapacity || stream_len < 0) return -1;
  const int32_t on = algo == BP_ALGO_PREFIX ? (kPrefixShared | kPrefixGlobal) : 0;
  return prefix_handles(d, c, stream_len * c, on) ? BP_ALGO_PREFIX : BP_ALGO_DIRECT;
}

int64_t bp_lb_param_count(int32_t d, int64_t c, int64_t *lo, int64_t *hi) {
  if (d < 0 || d >= kNumDff || c < 1 || c > kMaxCapacity) return -1;
  int64_t l, u;
  param_range(d, c, l, u);
  if (lo) *lo = l;
  if (hi) *hi = u;
  return u >= l ? u - l + 1 : 0;
}

int64_t bp_lb_selfcheck_division(uint32_t d_lo, uint32_t d_hi, uint32_t n_hi, int64_t samples) {
  if (d_lo < 1 || d_hi < d_lo || d_hi >= (1u << 31) || n_hi >= (1u << 31) || samples < 0) return -1;
  int64_t bad = 0;
  uint64_t x = 0x9E3779B97F4A7C15ull;  // splitmix64 state
  for (uint64_t d = d_lo; d <= d_hi; ++d) {
    const Div31 D = div31_make((uint32_t)d);
    for (uint64_t n = 0; n <= n_hi; ++n)
      bad += div31((uint32_t)(2 * n), D) != (uint32_t)(n / d);
    for (int64_t s = 0; s < samples; ++s) {
      x += 0x9E3779B97F4A7C15ull;
      uint64_t z = x;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const uint32_t n = (uint32_t)(z & 0x7FFFFFFFu);
      bad += div31(2u * n, D) != n / (uint32_t)d;
    }
  }
  return bad;
}

}  // extern "C"
