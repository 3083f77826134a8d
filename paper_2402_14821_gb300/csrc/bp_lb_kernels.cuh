// bp_lb_kernels.cuh -- the kernels of the DFF lower-bound check.
//
//   plan_kernel     per instance: validate, count (DFF, lambda-tile) tiles,
//                   exclusive scan into a tile table; resets the work counter.
//   eval_kernel     persistent CTAs pull tiles from an atomic counter; a tile
//                   is (instance, DFF, NT*T consecutive lambdas).  The CTA
//                   stages the instance's items into shared memory (building
//                   the reduced instance on the fly for search nodes),
//                   evaluates T lambdas per thread, reduces a packed
//                   (bound, -index) key over the block and folds it into the
//                   instance's slot with one 64-bit atomicMax; the last tile
//                   of an instance writes its outputs and clears the slot.
//   reduce_kernel   the reduction alone (one CTA per search node).
//   debug_kernel    per-(DFF, lambda) bounds for spot checks.
//
// Paper: Alg. 2 (what is computed), Alg. 4 and Sec. 4 "Implementation
// details" (parameters across threads, items in shared memory, block-level
// max then one global atomic max) and Sec. 3 / Fig. 3 (the reduction).
#pragma once

#include <cuda_runtime.h>

#include "../../include/bp_lb.h"
#include "bp_lb_core.cuh"
#include "bp_lb_eval.cuh"

namespace bplb {

constexpr int kChunk = 2048;          // stream positions staged per pass
constexpr int kListTop = kChunk + 8;  // list buffer length (small up, big down)
constexpr int kMaxNodeBins = 16384;   // on-chip bin-load table limit

enum SrcMode : int { kSrcRaggedI32 = 0, kSrcRaggedI64 = 1, kSrcNodes = 2 };

struct EvalArgs {
  int32_t B;
  // ragged reduced instances
  const int64_t *offsets;
  const void *sizes;
  const int64_t *capacity;
  const int64_t *bins;
  // search nodes
  int32_t num_base;
  const int64_t *base_offsets;
  const int32_t *base_sizes;
  const int64_t *base_capacity;
  const int32_t *node_base;
  const int64_t *assign_offsets;
  const int32_t *assign;
  int32_t max_bins;
  // outputs
  int64_t *out_bound;
  bp_argmax_t *out_argmax;
  uint8_t *out_feasible;
  // schedule / scratch
  const int64_t *tile_start;  // [B+1]; nullptr: one instance with single_tiles tiles
  int64_t single_tiles;
  int64_t single_c;
  int64_t single_k;
  int64_t single_n;
  unsigned long long *keys;   // [B] packed (bound, -index) maxima, zero between calls
  unsigned int *done;         // [B] finished-tile counters, zero between calls
  unsigned long long *work;   // [1] next tile (persistent mode), nullptr otherwise
  uint32_t one;               // always 1 (see add_if_ge in bp_lb_eval.cuh)
  int32_t prefix_on;          // kPrefixShared | kPrefixGlobal bits (0: no prefix-count kernel)
  const int64_t *ptile_start; // [B+1] prefix-kernel tile table, or nullptr (single instance)
  int64_t single_ptiles;
  unsigned long long *pwork;  // [1] next prefix tile (persistent mode)
  int64_t plpt;               // parameters per prefix-kernel tile
  int32_t vb2_on;             // route VB2 (c <= kVb2FixedCap) to the VB2 kernel
  int32_t pad_vb2;
  const int64_t *vtile_start; // [B+1] VB2-kernel tile table, or nullptr (single instance)
  int64_t single_vtiles;
  unsigned long long *vwork;  // [1] next VB2 tile (persistent mode)
  int32_t verdict;            // verdict-only mode (early exit, exact feasibility)
  uint32_t dff_off;           // bit d set: DFF d is left out of the bound (default 0: all six)
  int32_t *gscratch;          // prefix tables in global memory: kGlobalTableInts per CTA
  int32_t prune;              // skip parameters that provably cannot win (exact)
  int32_t pad_prune;
  // measurement (nullptr unless kernel timing is on): [0] VB2 (item,
  // parameter) pairs evaluated by the VB2 kernel, [1] by the generic kernel,
  // [2] VB2 parameters evaluated, [3] VB2 parameters pruned
  unsigned long long *work_count;
  // [B][8] per instance: n_small, n_big, n_half, n_full, sum_big w, sum w of
  // the reduced instance, written by the prefix kernel; [7] = 1 once written
  // (cleared by the plan kernel).  nullptr: not kept.
  long long *isums;
  // VB2 kernel tile length, chosen by the plan kernel (nullptr: kVb2LPT), and
  // the number of VB2 tiles it aims at
  long long *vlpt;
  int64_t vb2_target_tiles;
  // reduction variants of the search-node mode (transform_bins):
  // BP_REDUCE_LOADS or BP_REDUCE_CLOSE, and optional per-bin maximum loads
  // (node b's bin j: bin_max[bin_max_offsets[b] + j], 0 <= it <= c)
  int32_t reduce_mode;
  int32_t pad_reduce;
  const int64_t *bin_max_offsets;
  const int32_t *bin_max;
  // VB2's parameter cap of Sec. 4 (bp_lb_set_vb2_cap): per instance the
  // largest VB2 parameter evaluated, min(c, floor(UINT_MAX / (r max w'))),
  // written by vb2cap_kernel before the evaluation kernels; nullptr: VB2's
  // whole range [2, c].
  const int64_t *vb2_hi;
  // A window [g_lo, g_hi) of the flattened parameter index (bp_lb_eval_range):
  // with `windowed` set, the direct kernel's tiles cover only the parameters
  // inside it, and the finishing CTA also writes the packed key to out_key
  // (nullptr: not written).
  int32_t windowed;
  uint32_t g_lo, g_hi;
  int64_t *out_key;
  // The cluster kernel's unit table (tables in a cluster's distributed shared
  // memory, prefix_home 3): [B+1] exclusive prefix of units per instance, or
  // nullptr (single instance: single_ctiles units), and its work counter.
  const int64_t *ctile_start;
  int64_t single_ctiles;
  unsigned long long *cwork;
};

// Shared-memory budget of the prefix-count tables (bytes; 48 KB lets four
// CTAs share an SM), and the number of parameters per prefix-kernel tile for
// batches (long tiles amortise building the tables) and for a single check
// (short tiles spread it over more SMs).
constexpr int64_t kPrefixSmemBytes = 49152;
constexpr int64_t kPrefixLPTBatch = 16384;
constexpr int64_t kPrefixLPTSingle = 1024;

// Bytes of the prefix-count tables of DFF d at capacity c (0: not on that path):
// u-domain tables of (c - 1) / 2 + 2 entries (MT one, RAD2 two, CCM1 one) and
// the w-domain table of c + 2 entries (FS1, BJ1), all int32.
BPLB_HD int64_t prefix_table_bytes(int d, int64_t c) {
  const int64_t nu = (c - 1) / 2 + 2;
  switch (d) {
    case kMT:
    case kCCM1: return 4 * nu;
    case kRAD2: return 8 * nu;
    case kFS1:
    case kBJ1:  return 4 * (c + 2);
    default:    return 0;
  }
}

// prefix_on bits: the prefix-count kernel is on (its tables in shared
// memory where they fit), its tables may also live in a global-memory
// scratch of kGlobalTableInts int32 per CTA (L2-resident; for capacities up
// to about 2^20), and tables too large for one CTA but within
// kClusterTableInts may be spread over the shared memory of a thread-block
// cluster of kClusterCtas CTAs (the cluster kernel), kSliceInts int32 each:
// entry x lives in CTA x >> kSliceShift of the cluster.
constexpr int32_t kPrefixShared = 1;
constexpr int32_t kPrefixGlobal = 2;
constexpr int32_t kPrefixCluster = 4;
constexpr int64_t kGlobalTableInts = int64_t(1) << 20;
constexpr int kClusterCtas = 8;
constexpr int kSliceShift = 14;
constexpr int64_t kSliceInts = int64_t(1) << kSliceShift;
constexpr int64_t kClusterTableInts = kClusterCtas * kSliceInts;

// Where the prefix-count tables of DFF d of an instance with capacity c
// whose reduced sizes sum to at most sum_bound live: 0 nowhere (the direct
// kernels evaluate it), 1 one CTA's shared memory, 2 the global scratch (both
// the prefix kernel), 3 a cluster's shared memory (the cluster kernel).  The
// sums must fit 32 bits; FS1's count sum, at most 101 sum_bound / c, too.
BPLB_HD int table_home(int64_t bytes, int32_t on) {
  if (bytes <= kPrefixSmemBytes) return 1;
  if ((on & kPrefixCluster) && bytes <= 4 * kClusterTableInts) return 3;
  if ((on & kPrefixGlobal) && bytes <= 4 * kGlobalTableInts) return 2;
  return 0;
}

BPLB_HD int prefix_home(int d, int64_t c, int64_t sum_bound, int32_t on) {
  if (!(on & kPrefixShared) || sum_bound >= (int64_t(1) << 31)) return 0;
  if (d == kFS1 && sum_bound >= (int64_t(1) << 25) * c) return 0;  // sum_bound / c >= 2^25
  const int64_t bytes = prefix_table_bytes(d, c);
  if (bytes == 0) return 0;
  return table_home(bytes, on);
}

// The routing functions (prefix_home, prefix_u_merged and what calls them)
// depend on an instance's sum bound only through these three thresholds, so
// that instances of one capacity and class route alike (the routing caches
// of the planning and prefix kernels key on it).
BPLB_HD int route_class(int64_t c, int64_t sum_bound) {
  return (sum_bound < (int64_t(1) << 31) ? 1 : 0) | (sum_bound < (int64_t(1) << 25) * c ? 2 : 0) |
         (sum_bound < (int64_t(1) << 15) * c ? 4 : 0);
}

BPLB_HD bool prefix_handles(int d, int64_t c, int64_t sum_bound, int32_t on) {
  return prefix_home(d, c, sum_bound, on) != 0;
}

// Parameters per tile of the VB2 kernel: at least kVb2LPT; longer (up to
// kVb2MaxLPT, in multiples of 1024) when the batch has more than
// vb2_target_tiles tiles' worth, so that tiles pruned whole (they only pass
// through the scheduler) are few.
constexpr int64_t kVb2LPT = 4096;
constexpr int64_t kVb2MaxLPT = 65536;
constexpr int64_t kVb2TilesPerSm = 24;

// Which kernel evaluates DFF d of an instance: the prefix-count kernel
// (prefix_handles), the VB2 kernel (VB2 on its fixed-point path), or the
// generic direct kernel; none when the DFF is left out (dff_off).
// kRouteCluster only selects what route_tiles counts: the prefix-routed
// units whose tables are a cluster's (prefix_home 3).
enum : int { kRouteNone = -1, kRouteDirect = 0, kRoutePrefix = 1, kRouteVb2 = 2, kRouteCluster = 3 };

BPLB_HD int dff_kernel(int d, int64_t c, int64_t sum_bound, int32_t prefix_on, int32_t vb2_on,
                       uint32_t dff_off) {
  if ((dff_off >> d) & 1u) return kRouteNone;
  if (prefix_handles(d, c, sum_bound, prefix_on)) return kRoutePrefix;
  if (vb2_on && d == kVB2 && c <= kVb2FixedCap) return kRouteVb2;
  return kRouteDirect;
}

// Where the u group's tables (E plus packed counts, 8 bytes per u) live
// (prefix_home's numbering).
BPLB_HD int prefix_u_home(int64_t c, int32_t on) {
  return table_home(8 * ((c - 1) / 2 + 2), on);
}

// MT, RAD2 and CCM1 share one prefix-kernel tile per instance (the u group:
// one pass over the items builds E and a table of packed small/big counts)
// when at least two of them go to the prefix kernel, the two u-domain tables
// fit (shared memory, each member then within one tile of lpt parameters; or
// the global scratch), and the counts fit 16 bits (stream length below 2^15;
// sum_bound = stream length c).
BPLB_HD bool prefix_u_merged(int64_t c, int64_t sum_bound, int32_t prefix_on, int32_t vb2_on,
                             uint32_t dff_off, int64_t lpt) {
  if (!(prefix_on & kPrefixShared) || sum_bound >= (int64_t(1) << 15) * c) return false;
  const int home = prefix_u_home(c, prefix_on);
  if (home == 0) return false;
  const int ds[3] = {kMT, kRAD2, kCCM1};
  int members = 0;
  for (int i = 0; i < 3; ++i) {
    const int64_t pc = param_count(ds[i], c);
    if (pc == 0 || dff_kernel(ds[i], c, sum_bound, prefix_on, vb2_on, dff_off) != kRoutePrefix)
      continue;
    if (home == 1 && pc > lpt) return false;
    ++members;
  }
  return members >= 2;
}

// ceil(count / lpt) in 32 bits: counts are at most 2^30 + 1 and tile
// lengths at most 2^16 wherever tiles are counted.
BPLB_HD int64_t tile_count(int64_t count, int64_t lpt) {
  return (int64_t)(((uint32_t)count + (uint32_t)lpt - 1u) / (uint32_t)lpt);
}

// FS1 shares the first of BJ1's prefix-kernel tiles (both read the w-domain
// table) when both go to the prefix kernel; otherwise it has a tile of its own.
BPLB_HD bool prefix_w_merged(int64_t c, int64_t sum_bound, int32_t prefix_on, int32_t vb2_on,
                             uint32_t dff_off) {
  return dff_kernel(kFS1, c, sum_bound, prefix_on, vb2_on, dff_off) == kRoutePrefix &&
         dff_kernel(kBJ1, c, sum_bound, prefix_on, vb2_on, dff_off) == kRoutePrefix;
}

// Tiles of DFF d routed to the prefix-count tables: one when its tables are in
// the global scratch or a cluster's shared memory (built once per tile, so
// the tile takes the whole range), else ceil(count / lpt).
BPLB_HD int64_t prefix_dff_tiles(int d, int64_t c, int64_t sum_bound, int32_t on, int64_t lpt) {
  const int64_t pc = param_count(d, c);
  if (pc == 0) return 0;
  return prefix_home(d, c, sum_bound, on) >= 2 ? 1 : tile_count(pc, lpt);
}

// Tiles of one kernel for an instance: lpt parameters each, DFFs in paper
// order; with the prefix-count tables the u group, when merged, is one tile,
// and FS1 rides on BJ1's first tile when prefix_w_merged.  kRoutePrefix
// counts the prefix kernel's tiles (tables in a CTA's shared memory or the
// global scratch), kRouteCluster the cluster kernel's (prefix_home 3).
BPLB_HD int64_t route_tiles(int route, int64_t c, int64_t lpt, int64_t sum_bound, int32_t prefix_on,
                            int32_t vb2_on, uint32_t dff_off) {
  const bool cl = route == kRouteCluster;
  const bool pre = route == kRoutePrefix || cl;
  const bool merged = pre && prefix_u_merged(c, sum_bound, prefix_on, vb2_on, dff_off, lpt);
  const bool wmerged = pre && prefix_w_merged(c, sum_bound, prefix_on, vb2_on, dff_off);
  int64_t t = (merged && (prefix_u_home(c, prefix_on) == 3) == cl) ? 1 : 0;
  for (int d = 0; d < kNumDff; ++d) {
    if (merged && (d == kMT || d == kRAD2 || d == kCCM1)) continue;
    if (wmerged && d == kFS1) continue;
    if (dff_kernel(d, c, sum_bound, prefix_on, vb2_on, dff_off) != (pre ? kRoutePrefix : route))
      continue;
    if (!pre) {
      t += tile_count(param_count(d, c), lpt);
    } else if ((prefix_home(d, c, sum_bound, prefix_on) == 3) == cl) {
      t += cl ? (param_count(d, c) > 0 ? 1 : 0)
              : prefix_dff_tiles(d, c, sum_bound, prefix_on, lpt);
    }
  }
  return t;
}

// Instance view resolved per tile.
struct InstView {
  int64_t c, k;
  int64_t n;        // base items (nodes) or items (ragged)
  int64_t begin;    // ragged: offset of the first item
  const int32_t *w; // nodes: base sizes
  const int32_t *a; // nodes: assignment
};

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Programmatic dependent launch (the batched calls launch the prefix, VB2
// and generic kernels with programmatic stream serialization): a kernel
// waits for the grid before it in the stream to complete, its writes
// visible, before it reads anything that grid wrote (pdl_wait), and lets the
// grid after it be scheduled early (pdl_release), so that launch latency
// overlaps the previous kernel's tail.  Without the launch attribute both
// are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Verdict mode (Alg. 2's early exit): an instance is decided once its result
// slot holds a bound above k -- it is infeasible whatever the remaining
// parameters give.  Read by one thread; the caller broadcasts the answer.
__device__ __forceinline__ bool slot_decided(const unsigned long long *slot, int64_t k) {
  const unsigned long long key = *reinterpret_cast<const volatile unsigned long long *>(slot);
  return (int64_t)(key >> 32) > k;
}

// Calls f(i, x[i], y[i]) (ONE: f(i, x[i], 0)) for i in [0, n), over the
// CTA's NT threads, reading four consecutive entries with one 16-byte load
// wherever the arrays allow.  Thread t takes the groups of four entries that
// start on x's 16-byte boundaries (the first and last groups may be partial:
// their entries inside [0, n) are read one at a time); y, when given, is read
// alongside when it has the same 16-byte phase as x, else every entry is read
// on its own.  f has one call site, so a large f is compiled once.  With
// PARTS > 1 the groups are dealt over PARTS CTAs, this one being `part`.
template <int NT, bool ONE, int PARTS = 1, class F>
__device__ __forceinline__ void for_items_vec(const int32_t *x, const int32_t *y, int64_t n, F f,
                                              uint32_t part = 0u) {
  const int64_t px = (int64_t)((reinterpret_cast<uintptr_t>(x) >> 2) & 3u);
  const int64_t py = ONE ? px : (int64_t)((reinterpret_cast<uintptr_t>(y) >> 2) & 3u);
  const bool vec = px == py;
  const int64_t ph = vec ? px : 0;  // x's offset (entries) within its 16-byte line
  const int64_t ngroups = (n + ph + 3) >> 2;
  for (int64_t g = (int64_t)part * NT + threadIdx.x; g < ngroups; g += (int64_t)PARTS * NT) {
    const int64_t base = 4 * g - ph;  // entry index of the group's first value
    int4 vx = make_int4(0, 0, 0, 0), vy = vx;
    if (vec && base >= 0 && base + 3 < n) {
      vx = *reinterpret_cast<const int4 *>(x + base);
      if (!ONE) vy = *reinterpret_cast<const int4 *>(y + base);
    } else {
      if (base >= 0 && base < n) vx.x = x[base];
      if (base + 1 >= 0 && base + 1 < n) vx.y = x[base + 1];
      if (base + 2 >= 0 && base + 2 < n) vx.z = x[base + 2];
      if (base + 3 < n) vx.w = x[base + 3];
      if (!ONE) {
        if (base >= 0 && base < n) vy.x = y[base];
        if (base + 1 >= 0 && base + 1 < n) vy.y = y[base + 1];
        if (base + 2 >= 0 && base + 2 < n) vy.z = y[base + 2];
        if (base + 3 < n) vy.w = y[base + 3];
      }
    }
#pragma unroll 1
    for (int e = 0; e < 4; ++e) {
      const int64_t i = base + e;
      if (i < 0 || i >= n) continue;
      const int32_t xv = e == 0 ? vx.x : (e == 1 ? vx.y : (e == 2 ? vx.z : vx.w));
      const int32_t yv = e == 0 ? vy.x : (e == 1 ? vy.y : (e == 2 ? vy.z : vy.w));
      f(i, xv, ONE ? 0 : yv);
    }
  }
}

// Warp-aggregated append to a shared-memory list counter; returns the slot.
__device__ __forceinline__ int warp_append(bool pred, int *counter) {
  const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
  if (mask == 0) return -1;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if ((int)lane_id() == leader) base = atomicAdd(counter, __popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  return base + __popc(mask & ((1u << lane_id()) - 1u));
}

template <class V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = x > v ? x : v;
  }
  return v;
}

__device__ __forceinline__ void write_error(const EvalArgs &A, int64_t b) {
  if (A.out_key != nullptr) A.out_key[b] = -BP_ERANGE;
  A.out_bound[b] = -BP_ERANGE;
  if (A.out_argmax) {
    bp_argmax_t e;
    e.dff = -1;
    e.pad = 0;
    e.lambda = -1;
    A.out_argmax[b] = e;
  }
  if (A.out_feasible) A.out_feasible[b] = 0;
}

__device__ __forceinline__ void write_result(const EvalArgs &A, int64_t b, unsigned long long key,
                                             int64_t c, int64_t k) {
  const int64_t lb = (int64_t)(key >> 32);
  const uint32_t g = 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull);
  if (A.out_key != nullptr) A.out_key[b] = (int64_t)key;
  A.out_bound[b] = lb;
  if (A.out_argmax) {
    bp_argmax_t r;
    r.dff = -1;  // key 0: no parameter was evaluated
    r.lambda = -1;
    if (key != 0ull) unflatten(g, c, r.dff, r.lambda);
    r.pad = 0;
    A.out_argmax[b] = r;
  }
  if (A.out_feasible) A.out_feasible[b] = (uint8_t)(lb <= k);
}

// The parameters of DFF d that a call evaluates: its range [lo, hi], or with
// a window [g_lo, g_hi) of the flattened index only those whose index lies
// inside it (hi < lo when none).  Returns their number.
BPLB_HD int64_t window_range(int d, int64_t c, int32_t windowed, uint32_t g_lo, uint32_t g_hi,
                             int64_t &lo, int64_t &hi) {
  param_range(d, c, lo, hi);
  const int64_t n = hi >= lo ? hi - lo + 1 : 0;
  if (!windowed) return n;
  const int64_t off = flat_index(d, lo, c);  // index of the DFF's first parameter
  const int64_t a = max((int64_t)g_lo - off, (int64_t)0), e = min((int64_t)g_hi - off, n);
  if (e <= a) {
    hi = lo - 1;
    return 0;
  }
  hi = lo + e - 1;
  lo += a;
  return e - a;
}

// Last VB2 parameter of instance b: its range's upper end, or the cap of
// Sec. 4 when the handle has it on (vb2cap_kernel).
__device__ __forceinline__ int64_t vb2_last(const EvalArgs &A, int64_t b, int64_t hi_d) {
  return A.vb2_hi != nullptr ? min(hi_d, A.vb2_hi[b]) : hi_d;
}

// ---------------------------------------------------------------------------
// plan_kernel: one block.  Validates every instance, writes tile_start[0..B]
// (exclusive scan of tiles per instance; 0 tiles and an error result for an
// invalid one), clears keys/done and resets the work counter.
// ---------------------------------------------------------------------------
// Block-wide exclusive scan step of plan_kernel over Q quantities at once:
// excl[q] = the exclusive prefix of v[q] within this pass plus carry[q], and
// carry[q] advances by the pass total (four barriers for all Q).
template <int Q>
__device__ __forceinline__ void plan_scan(const int64_t (&v)[Q], int64_t (*s_warp)[32],
                                          int64_t *carry, int64_t (&excl)[Q]) {
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  const int nw = (int)(blockDim.x >> 5);
  int64_t x[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) x[q] = v[q];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x[q], o);
      if (lane >= o) x[q] += y;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int q = 0; q < Q; ++q) s_warp[q][warp] = x[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      int64_t wv = lane < nw ? s_warp[q][lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, wv, o);
        if (lane >= o) wv += y;
      }
      s_warp[q][lane] = wv;  // inclusive warp prefix
    }
  }
  __syncthreads();
  int64_t total[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    excl[q] = carry[q] + (warp ? s_warp[q][warp - 1] : 0) + x[q] - v[q];
    total[q] = s_warp[q][nw - 1];
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int q = 0; q < Q; ++q) carry[q] += total[q];
  __syncthreads();
}

// VB2's tile length: the batch's VB2 parameters over the target tile count,
// rounded up to a multiple of 1024, within [kVb2LPT, kVb2MaxLPT].
__device__ __forceinline__ int64_t plan_vlpt(const EvalArgs &A, int64_t vb2_params) {
  if (A.vlpt == nullptr || !A.vb2_on) return kVb2LPT;
  const int64_t tgt = max(A.vb2_target_tiles, (int64_t)1);
  const int64_t want = (vb2_params + tgt - 1) / tgt;
  return min(kVb2MaxLPT, max(kVb2LPT, (want + 1023) / 1024 * 1024));
}

// plan_kernel: one block.  Validates every instance and writes the tile
// tables of the direct kernel (tile_start[0..B]), of the prefix kernel
// (ptile_start[0..B]), of the cluster kernel (ctile_start[0..B]) and of the
// VB2 kernel (vtile_start[0..B]); an invalid instance gets no tiles and an
// error result.  Clears keys/done and resets
// the work counters.  Each thread takes kPlanPerThread consecutive instances
// (their tile counts summed locally, so that one block scan per quantity
// covers 1024 kPlanPerThread instances: the scans' barriers are most of the
// kernel's time) and keeps its last instance's routing, reused while the
// capacity and route class repeat (every node of a search-node batch).
constexpr int kPlanPerThread = 4;

// Stores a thread's K consecutive entries v[0..K) of out (from entry wb +
// K lane, wb the warp's first) so that each store instruction of the warp
// writes 32 consecutive entries: the warp's 32 K entries are transposed with
// shuffles (entry e of the block is lane e / K's v[e % K]).  Whole warps.
template <int K, typename T>
__device__ __forceinline__ void plan_store(T *out, int64_t wb, const T (&v)[K], int64_t B) {
  const int lane = (int)lane_id();
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = 32 * i + lane;
    T x = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T y = __shfl_sync(0xFFFFFFFFu, v[k], e / K);
      if (e % K == k) x = y;
    }
    if (wb + e < B) out[wb + e] = x;
  }
}

template <int MODE>
__global__ void __launch_bounds__(1024)
    plan_kernel(EvalArgs A, int64_t lpt, int64_t *tile_start, int64_t *ptile_start,
                int64_t *vtile_start, int64_t *ctile_start) {
  constexpr int K = kPlanPerThread;
  __shared__ int64_t s_warp[3][32];
  __shared__ int64_t s_carry[4];  // direct, prefix | cluster, VB2 parameters, VB2 tiles
  pdl_release();  // the prefix kernel's CTAs may be scheduled now; they wait for this grid
  // a batch of one pass also makes VB2's tile table in it (VB2's tile length
  // is known after its scan); larger ones in a second pass
  const bool one_pass = A.B <= (int64_t)blockDim.x * K;
  if (threadIdx.x == 0) {
    s_carry[0] = s_carry[1] = s_carry[2] = s_carry[3] = 0;
    *A.work = 0ull;
    if (A.pwork) *A.pwork = 0ull;
    if (A.cwork) *A.cwork = 0ull;
    if (A.vwork) *A.vwork = 0ull;
  }
  __syncthreads();
  // one pass over the instances: validate, count the direct and prefix tiles
  // and VB2's parameters (kept in vtile_start[b], low 32 bits, with the
  // instance's other tiles in the high 32, until the VB2 tile length is
  // known: VB2's parameters of the whole batch over the target tile count)
  // routing of capacity rc_c and route class rc_k; rc_p packs the prefix
  // kernel's tiles (low 32 bits) and the cluster kernel's units (high),
  // scanned together: a handful of each per instance, so neither field of a
  // batch's sum reaches 2^32
  int64_t rc_c = -1, rc_t = 0, rc_p = 0, rc_v = 0;
  int rc_k = -1;
  for (int64_t b0 = 0; b0 < A.B; b0 += (int64_t)blockDim.x * K) {
    const int64_t bt = b0 + (int64_t)threadIdx.x * K;  // this thread's first instance
    const int64_t wb = b0 + (int64_t)(threadIdx.x & ~31u) * K;  // its warp's first
    int64_t tiles[K], ptiles[K], pvs[K];
    int64_t st = 0, sp = 0, sv = 0;
    // the K instances' inputs first, with no store in between (a store could
    // alias them), so that their memory latencies overlap: the instance's
    // own fields, then those of a node's base instance
    bool okj[K];
    int64_t cj[K], Lj[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int64_t b = bt + j < A.B ? bt + j : A.B - 1;  // clamped: the result unused past B
      if (MODE == kSrcNodes) {
        const int32_t base = A.node_base[b];
        const int64_t na = A.assign_offsets[b + 1] - A.assign_offsets[b];
        const int64_t k = A.bins[b];
        okj[j] = base >= 0 && base < A.num_base && na >= 0 && k >= 0 && k <= A.max_bins &&
                 (A.bin_max == nullptr || A.bin_max_offsets[b + 1] - A.bin_max_offsets[b] == k);
        cj[j] = base;  // the base instance until its fields are read
        Lj[j] = na;
      } else {
        cj[j] = A.capacity[b];
        Lj[j] = A.offsets[b + 1] - A.offsets[b];
        okj[j] = A.bins[b] >= 0;
      }
    }
    if (MODE == kSrcNodes) {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int64_t b = bt + j < A.B ? bt + j : A.B - 1;
        const int32_t base = okj[j] ? (int32_t)cj[j] : 0;
        const int64_t c = okj[j] ? A.base_capacity[base] : 0;
        const int64_t n = okj[j] ? A.base_offsets[base + 1] - A.base_offsets[base] : 0;
        // a node's stream: its base instance's items and its bins' loads
        okj[j] = okj[j] && n == Lj[j] && n <= kMaxItems;
        cj[j] = c;
        Lj[j] = n + A.bins[b];
      }
    }
    // the key slots and sums flags of the pass's instances, coalesced
    for (int i = 0; i < K; ++i) {
      const int64_t b = b0 + threadIdx.x + (int64_t)blockDim.x * i;
      if (b < A.B) {
        A.keys[b] = 0ull;
        if (A.isums) A.isums[8 * b + 7] = 0;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int64_t b = bt + j;
      tiles[j] = ptiles[j] = pvs[j] = 0;
      if (b < A.B) {
        const int64_t c = cj[j], L = Lj[j];
        // (a node's n and k were checked above)
        const bool ok = okj[j] && c >= 1 && c <= kMaxCapacity &&
                        (MODE == kSrcNodes || (L >= 0 && L <= kMaxItems));
        if (ok) {
          const int rk = route_class(c, L * c);
          if (c != rc_c || rk != rc_k) {
            rc_t = route_tiles(kRouteDirect, c, lpt, L * c, A.prefix_on, A.vb2_on, A.dff_off);
            rc_p = route_tiles(kRoutePrefix, c, A.plpt, L * c, A.prefix_on, A.vb2_on, A.dff_off);
            if (ctile_start != nullptr && (A.prefix_on & kPrefixCluster))
              rc_p += route_tiles(kRouteCluster, c, A.plpt, L * c, A.prefix_on, A.vb2_on,
                                  A.dff_off) << 32;
            rc_v = (vtile_start != nullptr &&
                    dff_kernel(kVB2, c, L * c, A.prefix_on, A.vb2_on, A.dff_off) == kRouteVb2)
                       ? param_count(kVB2, c)
                       : 0;
            rc_c = c;
            rc_k = rk;
          }
          tiles[j] = rc_t;
          ptiles[j] = rc_p;
          pvs[j] = rc_v;
          // no parameter at all (only DFFs with an empty range left in): bound 0
          if (rc_t + rc_p + rc_v == 0) write_result(A, b, 0ull, c, A.bins[b]);
        } else {
          write_error(A, b);
        }
      }
      st += tiles[j];
      sp += ptiles[j];
      sv += pvs[j];
    }
    int64_t ex[3];
    {
      const int64_t sums[3] = {st, sp, sv};
      plan_scan<3>(sums, s_warp, s_carry, ex);
    }
    const int64_t e0 = ex[0], e1 = ex[1];
    int64_t v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = j ? v[j - 1] + tiles[j - 1] : e0;
    plan_store(tile_start, wb, v, A.B);
    if (ptile_start != nullptr || ctile_start != nullptr) {
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] = j ? v[j - 1] + ptiles[j - 1] : e1;
      if (ctile_start != nullptr) {
        int64_t u[K];
#pragma unroll
        for (int j = 0; j < K; ++j) u[j] = v[j] >> 32;
        plan_store(ctile_start, wb, u, A.B);
      }
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] &= 0xFFFFFFFFll;
      if (ptile_start != nullptr) plan_store(ptile_start, wb, v, A.B);
    }
    // the finished-tile counter starts at minus the instance's tiles
    // (instance_tiles); with a VB2 table, completed below once VB2's tile
    // length is known
#pragma unroll
    for (int j = 0; j < K; ++j)
      v[j] = tiles[j] + (ptiles[j] & 0xFFFFFFFFll) + (ptiles[j] >> 32);
    if (vtile_start != nullptr && one_pass) {
      // VB2's tiles now: the counter completed, the VB2 tile table written
      const int64_t vlpt = plan_vlpt(A, s_carry[2]);
      int64_t vt[K];
      int64_t svt = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        vt[j] = tile_count(pvs[j], vlpt);
        svt += vt[j];
      }
      int64_t e2[1];
      {
        const int64_t sums[1] = {svt};
        plan_scan<1>(sums, s_warp, &s_carry[3], e2);
      }
      uint32_t dn[K];
#pragma unroll
      for (int j = 0; j < K; ++j) dn[j] = 0u - (uint32_t)(v[j] + vt[j]);
      plan_store(A.done, wb, dn, A.B);
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] = j ? v[j - 1] + vt[j - 1] : e2[0];
      plan_store(vtile_start, wb, v, A.B);
    } else if (vtile_start != nullptr) {
#pragma unroll
      for (int j = 0; j < K; ++j) v[j] = pvs[j] | (v[j] << 32);
      plan_store(vtile_start, wb, v, A.B);
    } else {
      uint32_t dn[K];
#pragma unroll
      for (int j = 0; j < K; ++j) dn[j] = 0u - (uint32_t)v[j];
      plan_store(A.done, wb, dn, A.B);
    }
  }
  __syncthreads();
  const int64_t vlpt = plan_vlpt(A, s_carry[2]);
  if (threadIdx.x == 0 && A.vlpt != nullptr) *A.vlpt = vlpt;
  // a larger batch: the VB2 tile table from the kept parameter counts (each
  // thread rereads its own entries)
  if (vtile_start != nullptr && !one_pass) {
    for (int64_t b0 = 0; b0 < A.B; b0 += (int64_t)blockDim.x * K) {
      const int64_t bt = b0 + (int64_t)threadIdx.x * K;
      const int64_t wb = b0 + (int64_t)(threadIdx.x & ~31u) * K;
      int64_t vt[K];
      uint32_t tot[K];
      int64_t sv = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const int64_t pv = bt + j < A.B ? vtile_start[bt + j] : 0;
        vt[j] = tile_count(pv & 0xFFFFFFFFll, vlpt);
        tot[j] = (uint32_t)(pv >> 32);
        sv += vt[j];
      }
      // (every read of this pass's entries precedes the scan's barriers)
      int64_t e2[1];
      {
        const int64_t sums[1] = {sv};
        plan_scan<1>(sums, s_warp, &s_carry[3], e2);
      }
      int64_t v[K];
      uint32_t dn[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        v[j] = j ? v[j - 1] + vt[j - 1] : e2[0];
        dn[j] = 0u - (tot[j] + (uint32_t)vt[j]);
      }
      plan_store(vtile_start, wb, v, A.B);
      plan_store(A.done, wb, dn, A.B);
    }
  }
  if (threadIdx.x == 0) {
    tile_start[A.B] = s_carry[0];
    if (ptile_start) ptile_start[A.B] = s_carry[1] & 0xFFFFFFFFll;
    if (ctile_start) ctile_start[A.B] = s_carry[1] >> 32;
    if (vtile_start) vtile_start[A.B] = s_carry[3];
  }
}

// ---------------------------------------------------------------------------
// Tile processing.
// ---------------------------------------------------------------------------
struct TileShared {
  int ns, nb, err;
  int skip;     // verdict mode: the instance was decided before this tile
  int done_vb2;  // VB2 kernel: the instance's VB2 was evaluated on its u-group tile
  int stop[2];  // verdict mode: decided before group g (double-buffered by g & 1)
  long long kcut[2];  // VB2 pruning: the cut of group g (double-buffered by g & 1)
  int gskip[2];       // VB2 pruning: group g pruned whole
  unsigned long long wc[4];  // work counts of this CTA (EvalArgs::work_count)
  unsigned long long warp_key[32];
  long long sums[6];
  unsigned long long sumF[2];  // VB2 fixed point: sum of F over the small and big lists
  uint32_t minw;               // smallest unpacked size > 0 of a node (transform_bins)
};

// Fetches stream position q: returns true and the size when q is an item of
// the (reduced) instance, false for a filtered position (a packed item).
template <int MODE>
__device__ __forceinline__ bool fetch_item(const EvalArgs &A, const InstView &I, const uint32_t *s_load,
                                           int64_t q, int64_t &w) {
  if (MODE == kSrcRaggedI32) {
    w = reinterpret_cast<const int32_t *>(A.sizes)[I.begin + q];
    return true;
  } else if (MODE == kSrcRaggedI64) {
    w = reinterpret_cast<const int64_t *>(A.sizes)[I.begin + q];
    return true;
  } else {
    if (q < I.n) {
      w = I.w[q];
      return I.a[q] == -1;
    }
    w = s_load[q - I.n];
    return true;
  }
}

// Stream length of an instance: its items, or for a search node its base
// items (packed ones are filtered out) followed by its bin loads.
template <int MODE>
__device__ __forceinline__ int64_t stream_len(const InstView &I) {
  return MODE == kSrcNodes ? I.n + I.k : I.n;
}

// Upper bound on the sum of an instance's reduced sizes (its stream length
// times c), the quantity prefix_handles tests; plan_kernel uses the same.
template <int MODE>
__device__ __forceinline__ int64_t sum_bound(const InstView &I) {
  return stream_len<MODE>(I) * I.c;
}

// The finished-tile ticket target of instance b: a single instance's tiles
// over all kernels; 0 in a batch, whose plan kernel presets each instance's
// counter to minus its tiles, so that the last tile's ticket is 2^32 - 1.
__device__ __forceinline__ int64_t instance_tiles(const EvalArgs &A, int64_t b) {
  if (!A.tile_start) return A.single_tiles + A.single_ptiles + A.single_vtiles + A.single_ctiles;
  return 0;
}

// Block max of the threads' keys, one atomicMax into the instance's slot, and
// the finished-tile ticket: the CTA finishing the instance's last tile writes
// its outputs and clears the slot.  Thread 32 (warp 1) does the global part,
// with no barrier after it, so that its atomics' round trips overlap warp 0's
// search for the CTA's next tile (tile_publish); nothing it reads in shared
// memory is written again before the next tile's fold.
template <int NT>
__device__ void fold_and_finalize(const EvalArgs &A, int64_t b, unsigned long long best, bool err,
                                  int64_t ntiles, const InstView &I,
                                  unsigned long long *warp_key) {
  static_assert(NT >= 64, "the fold's global part runs on warp 1");
  const int tid = threadIdx.x;
  best = warp_max_u64(best);
  if (lane_id() == 0) warp_key[tid >> 5] = best;
  __syncthreads();
  if (tid == 32) {
    unsigned long long m = 0ull;
    for (int w = 0; w < NT / 32; ++w) m = warp_key[w] > m ? warp_key[w] : m;
    if (m && !err) atomicMax(&A.keys[b], m);
    __threadfence();
    const unsigned int ticket = atomicAdd(&A.done[b], 1u);
    if (ntiles > 0 ? (int64_t)ticket == ntiles - 1 : ticket == 0xFFFFFFFFu) {
      __threadfence();
      const unsigned long long key = atomicExch(&A.keys[b], 0ull);
      A.done[b] = 0u;
      if (err) write_error(A, b);
      else write_result(A, b, key, I.c, I.k);
    }
  }
}

// Bin loads of a search node into s_load (read back by
// fetch_item); sets *err for a bad assignment or an overfull bin.
// Reduction variants (search-node mode; not in the paper, which reduces a
// bin to one item of its packed load, Fig. 3): a bin with maximum load
// cap_j < c becomes an item of load + c - cap_j (the capacity it cannot use
// is filled), and under BP_REDUCE_CLOSE a bin whose free space is below the
// smallest unpacked item of nonzero size (minw; all bins when there is none)
// becomes an item of size c.  Any completion of the partial packing still
// fits the reduced instance in the k bins, so every bound stays valid.
// Rewrites the bin loads s_load[0 .. k) in place; a cap outside [0, c] or
// below the bin's load sets *err.
template <int NT>
__device__ __forceinline__ void transform_bins(const EvalArgs &A, int64_t b, const InstView &I,
                                               uint32_t *s_load, uint32_t minw, int *err) {
  const int32_t *cap = A.bin_max != nullptr ? A.bin_max + A.bin_max_offsets[b] : nullptr;
  for (int64_t j = threadIdx.x; j < I.k; j += NT) {
    int64_t v = s_load[j];
    if (cap != nullptr) {
      const int32_t m = cap[j];
      if (m < 0 || (int64_t)m > I.c || v > (int64_t)m) {
        *err = 1;
        continue;
      }
      v += I.c - m;
    }
    if (A.reduce_mode == BP_REDUCE_CLOSE && v > 0 && I.c - v < (int64_t)minw) v = I.c;
    s_load[j] = (uint32_t)v;
  }
}

__device__ __forceinline__ bool bins_transformed(const EvalArgs &A) {
  return A.reduce_mode != BP_REDUCE_LOADS || A.bin_max != nullptr;
}

// Bin loads of search node b in shared memory (the reduction of Fig. 3, with
// the variants of transform_bins); *minw is scratch for the smallest unpacked
// size.  The caller synchronises before reading s_load.
template <int NT, int MODE>
__device__ __forceinline__ void node_loads(const EvalArgs &A, int64_t b, const InstView &I,
                                           uint32_t *s_load, uint32_t *minw, int *err) {
  if (MODE == kSrcNodes) {
    const bool tr = bins_transformed(A);
    for (int64_t j = threadIdx.x; j < I.k; j += NT) s_load[j] = 0u;
    if (tr && threadIdx.x == 0) *minw = 0xFFFFFFFFu;
    __syncthreads();
    for_items_vec<NT, false>(I.a, I.w, I.n, [&](int64_t, int32_t a, int32_t w) {
      if (w < 0 || (int64_t)w > I.c || a < -1 || (int64_t)a >= I.k) {
        *err = 1;
      } else if (a >= 0) {
        const uint32_t old = atomicAdd(&s_load[a], (uint32_t)w);
        if ((int64_t)old + w > I.c) *err = 1;
      } else if (tr && w > 0) {
        atomicMin(minw, (uint32_t)w);
      }
    });
    if (tr) {
      __syncthreads();
      transform_bins<NT>(A, b, I, s_load, *minw, err);
    }
  }
}

// Local (per-thread) instance sums, reduced over the block once per tile.
struct LocalSums {
  int64_t v[6];  // n_small, n_big, n_half, n_full, sumw_big, sumw
};

// Stages stream positions [p, p + len) into the shared lists (and, with
// `count`, adds the instance sums into S.sums):
//   ULIST: small items as u = w from index 0 up, big items as u = c - w from
//          kListTop - 1 down, each stored as u << shift (plus fl(u / c) in
//          s_a when stage_a);
//   else:  every nonzero item as w << shift from index 0 up.
// Sizes outside [0, c] set S.err.  `count` adds the instance sums.
template <int NT, int MODE, bool ULIST>
__device__ __forceinline__ void stage_chunk(const EvalArgs &A, const InstView &I, const uint32_t *s_load,
                                            int64_t p, int len, bool stage_a, bool fixed, bool count,
                                            int shift, uint32_t *s_items, float *s_a, TileShared &S) {
  const int64_t c = I.c;
  LocalSums ls;
#pragma unroll
  for (int e = 0; e < 6; ++e) ls.v[e] = 0;
  uint64_t fs = 0, fb = 0;  // sums of the fixed-point values (fixed only)
  for (int o = 0; o < len; o += NT) {
    const int64_t q = p + o + threadIdx.x;
    int64_t w = 0;
    bool have = false;
    if (o + (int)threadIdx.x < len) have = fetch_item<MODE>(A, I, s_load, q, w);
    if (have && (w < 0 || w > c)) {
      S.err = 1;
      have = false;
    }
    if (have && w == 0) have = false;
    if (count && have) ls.v[5] += w;
    if (ULIST) {
      const bool full = have && w == c;
      const bool small = have && !full && 2 * w < c;
      const bool big = have && !full && 2 * w > c;
      if (count) {
        ls.v[0] += small;
        ls.v[1] += big;
        ls.v[2] += have && 2 * w == c;
        ls.v[3] += full;
        if (big) ls.v[4] += w;
      }
      const int ps = warp_append(small, &S.ns);
      const int pb = warp_append(big, &S.nb);
      if (small) {
        if (fixed) {
          const uint32_t F = vb2_fixed_frac((uint64_t)w, (uint64_t)c);
          s_items[ps] = F;
          fs += F;
        } else {
          s_items[ps] = (uint32_t)w << shift;
        }
        if (stage_a) s_a[ps] = __fdiv_rn((float)w, (float)c);
      }
      if (big) {
        const int slot = kListTop - 1 - pb;
        if (fixed) {
          const uint32_t F = vb2_fixed_frac((uint64_t)(c - w), (uint64_t)c);
          s_items[slot] = F;
          fb += F;
        } else {
          s_items[slot] = (uint32_t)(c - w) << shift;
        }
        if (stage_a) s_a[slot] = __fdiv_rn((float)(c - w), (float)c);
      }
    } else {
      const int ps = warp_append(have, &S.ns);
      if (have) s_items[ps] = (uint32_t)w << shift;
    }
  }
  if (fixed) {
    fs = warp_sum(fs);
    fb = warp_sum(fb);
    if (lane_id() == 0) {
      if (fs) atomicAdd(&S.sumF[0], (unsigned long long)fs);
      if (fb) atomicAdd(&S.sumF[1], (unsigned long long)fb);
    }
  }
  // the instance sums go to shared memory now, so that no register holds
  // them through the evaluation
  if (count) {
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const long long x = warp_sum((long long)ls.v[e]);
      if (lane_id() == 0 && x != 0) atomicAdd((unsigned long long *)&S.sums[e], (unsigned long long)x);
    }
  }
}

// VB2 pruning (exact).  A VB2 parameter whose bound is at most kcut is
// skipped: in verdict mode kcut = k (it cannot make the instance infeasible);
// in full mode kcut comes from the instance's best key so far, B (read from
// its slot; it only grows): B when that key's flattened index precedes VB2's
// (a tie then loses to it), else B - 1 -- a skipped parameter is then below
// the final maximum or ties it behind an earlier parameter.  -1: no cut.
__device__ __forceinline__ long long vb2_cut(const unsigned long long *slot, uint32_t gbase) {
  const unsigned long long key = *reinterpret_cast<const volatile unsigned long long *>(slot);
  if (key == 0ull) return -1;
  const long long B = (long long)(key >> 32);
  const uint32_t g = 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull);
  return g < gbase ? B : B - 1;
}

// Whether VB2 parameter l may have a bound above kk (false proves lb <= kk).
// With ceil(x) < x + 1 for the small list and ceil(x) >= x for the big one,
// acc <= floor(X / c), X = l D + n_small (c - 1), D = sum_small u - sum_big u,
// and lb <= kk whenever S(acc) <= 2 kk (l - 1), i.e. floor(X / c) <= M with
// M = floor(((l - 1)(2 kk - K) + 2 n_small - 2 n_big) / 2),
// K = 2 n_big + n_half + 2 n_full (vb2_sum in bp_lb_core.cuh).  kk is at most
// the stream length L (every VB2 bound is at most L), so up to c = 65535 all
// of it fits 64 bits; larger capacities use 128.
__device__ __forceinline__ bool vb2_may_exceed(int64_t l, int64_t kk, int64_t c, int64_t Dd,
                                               int64_t ns, int64_t nb, int64_t K) {
  if (c <= kVb2FixedCap) {
    const int64_t M = ((l - 1) * (2 * kk - K) + 2 * ns - 2 * nb) >> 1;
    return l * Dd + ns * (c - 1) > (M + 1) * c - 1;
  }
  const __int128 M = ((__int128)(l - 1) * (2 * kk - K) + 2 * ns - 2 * nb) >> 1;
  return (__int128)l * Dd + (__int128)ns * (c - 1) > (M + 1) * (__int128)c - 1;
}

// Whether some VB2 parameter in [l0, l1] may have a bound above kk (kk <= L).
// vb2_may_exceed(l) implies G(l) > 0 with
// G(l) = 2 X(l) - c (Y(l) + 1) + 2, Y(l) = (l - 1)(2 kk - K) + 2 n_small - 2 n_big
// (M = floor(Y / 2) >= (Y - 1) / 2), and G is linear in l: G <= 0 at both ends
// rules out the whole range.  64-bit up to c = 65535, 128-bit above.
__device__ __forceinline__ bool vb2_range_may_exceed(int64_t l0, int64_t l1, int64_t kk, int64_t c,
                                                     int64_t Dd, int64_t ns, int64_t nb,
                                                     int64_t K) {
  if (c <= kVb2FixedCap) {
    auto G = [&](int64_t l) {
      const int64_t X = l * Dd + ns * (c - 1);
      const int64_t Y = (l - 1) * (2 * kk - K) + 2 * ns - 2 * nb;
      return 2 * X - c * (Y + 1) + 2;
    };
    return G(l0) > 0 || G(l1) > 0;
  }
  auto G = [&](int64_t l) {
    const __int128 X = (__int128)l * Dd + (__int128)ns * (c - 1);
    const __int128 Y = (__int128)(l - 1) * (2 * kk - K) + 2 * ns - 2 * nb;
    return 2 * X - (__int128)c * (Y + 1) + 2;
  };
  return G(l0) > 0 || G(l1) > 0;
}

// Whether a VB2 tile [l0, l1] of instance b can be skipped before anything is
// staged: VB2 was evaluated on the instance's u-group table (the prefix or
// cluster kernel published flag 2), or the instance's class counts and sums
// that they published (EvalArgs::isums, flag 1) and its cut -- k in verdict
// mode, else from its best key so far (vb2_cut) -- show that no parameter of
// the tile can change the result.  Thread 0 only.
__device__ __forceinline__ bool vb2_tile_pruned(const EvalArgs &A, int64_t b, int64_t c, int64_t k,
                                                int64_t L, int64_t l0, int64_t l1,
                                                uint32_t gbase) {
  if (A.isums == nullptr || !(A.verdict || A.prune) || l1 < l0) return false;
  const volatile long long *is = A.isums + 8 * b;
  const long long flag = is[7];
  if (flag == 2) return true;
  if (flag != 1) return false;
  __threadfence();
  const int64_t cut = A.verdict ? k : (int64_t)vb2_cut(&A.keys[b], gbase);
  if (cut < 0) return false;
  const int64_t ns = is[0], nb = is[1], nh = is[2], nf = is[3], swb = is[4], sw = is[5];
  const int64_t Dd = (sw - swb - nh * (c / 2) - nf * c) - (nb * c - swb);
  const int64_t K = 2 * nb + nh + 2 * nf;
  return !vb2_range_may_exceed(l0, l1, min(cut, L), c, Dd, ns, nb, K);
}

// Work counters of a CTA (measurement only): cleared at the kernel's start,
// added to EvalArgs::work_count once at its end.
__device__ __forceinline__ void work_count_begin(const EvalArgs &A, TileShared &S) {
  if (A.work_count != nullptr && threadIdx.x < 4) S.wc[threadIdx.x] = 0ull;
}

__device__ __forceinline__ void work_count_flush(const EvalArgs &A, TileShared &S) {
  if (A.work_count == nullptr) return;
  __syncthreads();
  if (threadIdx.x < 4 && S.wc[threadIdx.x] != 0ull)
    atomicAdd(&A.work_count[threadIdx.x], S.wc[threadIdx.x]);
}

// Evaluates one tile of DFF D: lambdas [lam0, lam_end) in groups of NT * T,
// thread t taking the T consecutive lambdas lam_g + t * T + j (j < T) of group
// g, so that the threads past the end of a short range form whole idle warps.  Returns the
// thread's largest key make_key(lb, flat index); 0 if it had no parameter.
// With DEBUG the thread's single parameter comes from a request list and its
// bound is written to req_out instead.
template <int NT, int T, int D, int MODE, bool DEBUG, bool VB2_FIXED_ONLY = false>
__device__ unsigned long long tile_dff(const EvalArgs &A, const InstView &I, int64_t lam0,
                                       int64_t lam_end, uint32_t *s_items, float *s_a,
                                       const uint32_t *s_load, TileShared &S,
                                       const int64_t *req_lam = nullptr, int64_t *req_out = nullptr,
                                       int64_t req_idx = -1,
                                       unsigned long long *vslot = nullptr,
                                       unsigned long long *kslot = nullptr) {
  constexpr bool ULIST = (D == kMT || D == kRAD2 || D == kCCM1 || D == kVB2);
  constexpr int GW = NT * T;
  const int tid = threadIdx.x;
  const int64_t c = I.c;
  int64_t lo_d, hi_d;
  param_range(D, c, lo_d, hi_d);
  const uint32_t gbase = flat_index(D, lo_d, c);
  // VB2_FIXED_ONLY: the caller guarantees c <= kVb2FixedCap (the other VB2
  // paths are compiled out of that instantiation)
  const bool vb2_fixed = (D == kVB2) && (VB2_FIXED_ONLY || c <= kVb2FixedCap);
  const bool stage_a = (D == kVB2) && !VB2_FIXED_ONLY && !vb2_fixed && c <= kVb2FloatCap;
  const uint32_t Y0 = vb2_fixed ? vb2_fixed_frac((uint64_t)c - 1, (uint64_t)c) : 0u;
  const bool narrow = c <= kNarrowCap;  // BJ1: terms < 2c stay below 2^30
  const bool fs1_fast = c <= kFs1FastCap;
  const bool ccm1_noshift = c <= kCcm1NoShiftCap;
  const bool bj1_noshift = c <= kBj1NoShiftCap;
  // stored value: u or w itself where the kernel divides it without a shift
  // (or compares it to raw thresholds), else doubled
  const int shift = (D == kFS1 || (D == kCCM1 && ccm1_noshift) || (D == kBJ1 && bj1_noshift)) ? 0 : 1;
  const Div31 Dc = div31_make((uint32_t)c);
  const uint32_t c2 = (uint32_t)(2 * c);

  const int64_t L = stream_len<MODE>(I);
  const bool one_chunk = L <= kChunk;
  const int ngroups = DEBUG ? 1 : (int)((lam_end - lam0 + GW - 1) / GW);
  unsigned long long best = 0ull;

  // VB2 pruning against the instance's best key so far (full mode)
  const bool kprune = D == kVB2 && !DEBUG && kslot != nullptr;
  for (int g = 0; g < ngroups; ++g) {
    // verdict mode: stop once another tile (or an earlier group) decided the
    // instance; full mode: this group's VB2 cut
    if ((vslot != nullptr || kprune) && g > 0) {
      if (tid == 0) {
        if (vslot != nullptr) S.stop[g & 1] = slot_decided(vslot, I.k) ? 1 : 0;
        if (kprune) S.kcut[g & 1] = vb2_cut(kslot, gbase);
        // the whole group pruned (vb2_range_may_exceed; the instance sums are
        // complete after the first group)
        S.gskip[g & 1] = 0;
        if (D == kVB2 && !S.err) {
          const int64_t cut = vslot != nullptr ? I.k : (int64_t)S.kcut[g & 1];
          if (cut >= 0) {
            const int64_t ns_ = S.sums[0], nb_ = S.sums[1], nh_ = S.sums[2], nf_ = S.sums[3];
            const int64_t swb = S.sums[4], sw = S.sums[5];
            const int64_t Dd = (sw - swb - nh_ * (c / 2) - nf_ * c) - (nb_ * c - swb);
            const int64_t K = 2 * nb_ + nh_ + 2 * nf_;
            const int64_t gl0 = lam0 + (int64_t)g * GW;
            const int64_t gl1 = min(lam_end, gl0 + GW) - 1;
            if (!vb2_range_may_exceed(gl0, gl1, min(cut, L), c, Dd, ns_, nb_, K)) {
              S.gskip[g & 1] = 1;
              if (A.work_count != nullptr) atomicAdd(&S.wc[3], (unsigned long long)(gl1 - gl0 + 1));
            }
          }
        }
      }
      __syncthreads();
      if (vslot != nullptr && S.stop[g & 1]) break;
      if (S.gskip[g & 1]) continue;
    }
    // ---- this group's parameters and their constants -------------------------
    int64_t lam[T];
    bool valid[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
      int64_t l;
      if (DEBUG) {
        l = (j == 0 && req_idx >= 0) ? req_lam[req_idx] : lo_d;
      } else {
        l = lam0 + (int64_t)g * GW + (int64_t)tid * T + j;
      }
      valid[j] = DEBUG ? (j == 0 && req_idx >= 0 && l >= lo_d && l <= hi_d) : (l < lam_end);
      lam[j] = valid[j] ? l : lo_d;
    }
    uint32_t k0[T], k1[T], k2[T];
    float kf[T];
    Div31 Dl[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
      const uint32_t l32 = (uint32_t)lam[j];
      k0[j] = k1[j] = k2[j] = 0;
      kf[j] = 0.f;
      Dl[j].m = Dl[j].l = 0;
      if (D == kMT) {
        k0[j] = 2u * l32;
      } else if (D == kRAD2) {
        k0[j] = 2u * l32;
        k1[j] = (uint32_t)(2 * c - 4 * lam[j]);
      } else if (D == kFS1) {
        k0[j] = 2u * l32 + 2u;
      } else if (D == kCCM1) {
        if (ccm1_noshift) k0[j] = div_noshift_make(l32);
        else Dl[j] = div31_make(l32);
      } else if (D == kVB2) {
        k0[j] = l32;
        kf[j] = (float)l32;
      } else {  // BJ1
        const uint32_t cm = (uint32_t)c - ((uint32_t)c / l32) * l32;  // c mod l
        if (bj1_noshift) {
          k0[j] = div_noshift_make(l32);
          k1[j] = l32;
          k2[j] = cm;
        } else {
          Dl[j] = div31_make(l32);
          k0[j] = 2u * l32;
          k1[j] = 2u * cm;
        }
      }
    }
    int64_t acc[T];
    int32_t n1[T];
    uint32_t n2s[T], n2b[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
      acc[j] = 0;
      n1[j] = 0;
      n2s[j] = n2b[j] = 0;
    }

    // ---- stream the instance through shared memory ---------------------------
    for (int64_t p = 0; p < L || (p == 0 && L == 0); p += kChunk) {
      const bool stage = (g == 0) || !one_chunk;
      if (stage) {
        if (tid == 0) {
          S.ns = 0;
          S.nb = 0;
          S.sumF[0] = S.sumF[1] = 0ull;
          if (kprune && g == 0) S.kcut[0] = vb2_cut(kslot, gbase);
        }
        if (g == 0 && p == 0 && tid < 6) S.sums[tid] = 0;
        __syncthreads();
        const int len = (int)min((int64_t)kChunk, L - p);
        stage_chunk<NT, MODE, ULIST>(A, I, s_load, p, len, stage_a, vb2_fixed, g == 0, shift,
                                     s_items, s_a, S);
        __syncthreads();
        const int ns = S.ns, nb = S.nb;
        const int ns_pad = (ns + 3) & ~3;
        const int bstart = (kListTop - nb) & ~3;
        if (tid < 4) {
          if (ns + tid < ns_pad) {
            s_items[ns + tid] = 0u;
            if (stage_a) s_a[ns + tid] = 0.f;
          }
          if (ULIST && bstart + tid < kListTop - nb) {
            s_items[bstart + tid] = 0u;
            if (stage_a) s_a[bstart + tid] = 0.f;
          }
        }
        __syncthreads();
      }
      int nv_before = 0;
#pragma unroll
      for (int j = 0; j < T; ++j) nv_before += valid[j] ? 1 : 0;
      // VB2 pruning (vb2_cut, vb2_may_exceed): parameters that cannot exceed
      // the cut are dropped, and a warp left with none skips the items.  The
      // instance sums are complete once the first pass over the stream is.
      if (D == kVB2 && (vslot != nullptr || kprune) && (one_chunk || g > 0) && !S.err) {
        const int64_t cut = vslot != nullptr ? I.k : (int64_t)S.kcut[g & 1];
        if (cut >= 0) {
          const int64_t ns_ = S.sums[0], nb_ = S.sums[1], nh_ = S.sums[2], nf_ = S.sums[3];
          const int64_t swb = S.sums[4], sw = S.sums[5];
          const int64_t Dd = (sw - swb - nh_ * (c / 2) - nf_ * c) - (nb_ * c - swb);
          const int64_t K = 2 * nb_ + nh_ + 2 * nf_;
          const int64_t kk = min(cut, L);
#pragma unroll
          for (int j = 0; j < T; ++j)
            valid[j] = valid[j] && vb2_may_exceed(lam[j], kk, c, Dd, ns_, nb_, K);
          bool mine = false;
#pragma unroll
          for (int j = 0; j < T; ++j) mine |= valid[j];
          if (!__any_sync(0xFFFFFFFFu, mine)) {
#pragma unroll
            for (int j = 0; j < T; ++j) valid[j] = false;
          }
        }
      }
      if (D == kVB2 && !DEBUG && A.work_count != nullptr && !S.err) {
        int nv = 0;
#pragma unroll
        for (int j = 0; j < T; ++j) nv += valid[j] ? 1 : 0;
        const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)nv);
        const uint32_t totb = __reduce_add_sync(0xFFFFFFFFu, (uint32_t)nv_before);
        if (lane_id() == 0) {
          if (tot != 0u)
            atomicAdd(&S.wc[VB2_FIXED_ONLY ? 0 : 1],
                      (unsigned long long)tot * (unsigned long long)(S.ns + S.nb));
          if (p == 0) {
            atomicAdd(&S.wc[2], (unsigned long long)tot);
            atomicAdd(&S.wc[3], (unsigned long long)(totb - tot));
          }
        }
      }
      bool any_valid = false;
#pragma unroll
      for (int j = 0; j < T; ++j) any_valid |= valid[j];
      if (!S.err && any_valid) {
        const int ns_pad = (S.ns + 3) & ~3;
        const int bstart = (kListTop - S.nb) & ~3;
        if (D == kMT) {
          const int K = group_len(c - 1);  // terms u2 < c
          uint64_t a64[T];
#pragma unroll
          for (int j = 0; j < T; ++j) a64[j] = 0;
          mt_list<T, false>(s_items, 0, ns_pad, K, k0, A.one, a64);
          mt_list<T, true>(s_items, bstart, kListTop, K, k0, A.one, a64);
#pragma unroll
          for (int j = 0; j < T; ++j) acc[j] += (int64_t)a64[j];
        } else if (D == kRAD2) {
          rad2_list<T, 1>(s_items, 0, ns_pad, k0, k1, A.one, n1, n2s);
          rad2_list<T, -1>(s_items, bstart, kListTop, k0, k1, A.one, n1, n2b);
        } else if (D == kFS1) {
          if (fs1_fast) fs1_list<T>(s_items, 0, ns_pad, group_len(c), k0, Dc, c2, c, acc);
          else fs1_list_wide<T>(s_items, 0, ns_pad, lam, c, acc);
        } else if (D == kCCM1) {
          const int K = group_len(c / 2);  // terms floor(u / l) <= c / 2
          if (ccm1_noshift) {
            ccm1_list_noshift<T, 1>(s_items, 0, ns_pad, K, k0, acc);
            ccm1_list_noshift<T, -1>(s_items, bstart, kListTop, K, k0, acc);
          } else {
            ccm1_list<T, 1>(s_items, 0, ns_pad, K, Dl, acc);
            ccm1_list<T, -1>(s_items, bstart, kListTop, K, Dl, acc);
          }
        } else if (D == kVB2) {
          const int K = group_len(c / 2 + 1);
          if (vb2_fixed) {
            vb2_list_fixed<T, 1>(s_items, 0, ns_pad, k0, Y0, S.sumF[0], acc);
            vb2_list_fixed<T, -1>(s_items, bstart, kListTop, k0, Y0, S.sumF[1], acc);
          } else if (VB2_FIXED_ONLY) {
            // unreachable: c <= kVb2FixedCap
          } else if (stage_a) {
            const uint32_t K2 = 0u - c2 * kF32RoundBits;
            vb2_list_float<T, 1>(s_items, s_a, 0, ns_pad, K, k0, kf, c2, K2, acc);
            vb2_list_float<T, -1>(s_items, s_a, bstart, kListTop, K, k0, kf, c2, K2, acc);
          } else {
            vb2_list_wide<T, 1>(s_items, 0, ns_pad, lam, c, acc);
            vb2_list_wide<T, -1>(s_items, bstart, kListTop, lam, c, acc);
          }
        } else {  // BJ1
          if (bj1_noshift) bj1_list_noshift<T>(s_items, 0, ns_pad, group_len(c), k0, k1, k2, acc);
          else if (narrow) bj1_list<T>(s_items, 0, ns_pad, group_len(2 * c), Dl, k0, k1, acc);
          else bj1_list_wide<T>(s_items, 0, ns_pad, lam, c, acc);
        }
      }
      if (!one_chunk) __syncthreads();
      if (L == 0) break;
    }

    // the instance sums are complete after the first pass over the stream
    if (g == 0 && !one_chunk) __syncthreads();
    if (S.err) break;
    InstSums sums;
    sums.n_small = S.sums[0];
    sums.n_big = S.sums[1];
    sums.n_half = S.sums[2];
    sums.n_full = S.sums[3];
    sums.sumw_big = S.sums[4];
    sums.sumw = S.sums[5];

    // ---- bounds of this group's parameters -----------------------------------------
#pragma unroll
    for (int j = 0; j < T; ++j) {
      if (!valid[j]) continue;
      const int64_t l = lam[j];
      const int64_t q = (D == kCCM1 || D == kBJ1) ? (int64_t)((uint32_t)c / (uint32_t)l) : 0;
      int64_t Ssum;
      if (D == kMT) Ssum = mt_sum(sums, c, (uint64_t)acc[j]);
      else if (D == kRAD2) Ssum = rad2_sum(sums, c, n1[j], n2s[j], n2b[j]);
      else if (D == kFS1) Ssum = fs1_sum(acc[j]);
      else if (D == kCCM1)
        Ssum = ccm1_sum(sums, q,
                        acc[j] + ((ccm1_noshift && l == 1) ? sums.n_small - sums.n_big : 0));
      else if (D == kVB2) Ssum = vb2_sum(sums, l, acc[j]);
      else Ssum = bj1_sum(sums, acc[j]);
      const int64_t lb = ceil_div_fast(Ssum, dff_at_c_q(D, l, c, q));
      if (DEBUG) {
        req_out[req_idx] = lb;
      } else {
        const unsigned long long key = make_key(lb, gbase + (uint32_t)(l - lo_d));
        best = key > best ? key : best;
      }
    }
    // verdict mode: publish a bound above k at once, so that other tiles stop
    if (vslot != nullptr && (int64_t)(best >> 32) > I.k) atomicMax(vslot, best);
  }
  return best;
}

// One tile: resolves its DFF and lambda range, computes the bin loads of a
// search node, runs tile_dff, then folds the block's best key into the
// instance slot; the last tile of the instance writes the outputs.
template <int NT, int T, int G, int MODE>
__device__ void process_tile(const EvalArgs &A, int64_t b, int64_t lt, int64_t ntiles,
                             const InstView &I, uint32_t *s_items, float *s_a, uint32_t *s_load,
                             TileShared &S) {
  constexpr int64_t LPT = (int64_t)NT * T * G;
  const int tid = threadIdx.x;
  const int64_t c = I.c;
  int d = 0;
  int64_t rem = lt;
  const int64_t sb = sum_bound<MODE>(I);
  int64_t lo_d, hi_d;
  for (d = 0; d < kNumDff; ++d) {
    if (dff_kernel(d, c, sb, A.prefix_on, A.vb2_on, A.dff_off) != kRouteDirect) continue;
    const int64_t nt =
        (window_range(d, c, A.windowed, A.g_lo, A.g_hi, lo_d, hi_d) + LPT - 1) / LPT;
    if (rem < nt) break;
    rem -= nt;
  }
  window_range(d, c, A.windowed, A.g_lo, A.g_hi, lo_d, hi_d);
  if (d == kVB2) hi_d = vb2_last(A, b, hi_d);
  const int64_t lam0 = lo_d + rem * LPT;
  const int64_t lam_end = max(lam0, min(hi_d + 1, lam0 + LPT));

  unsigned long long *vslot = A.verdict ? &A.keys[b] : nullptr;
  if (tid == 0) {
    S.err = 0;
    S.skip = (vslot != nullptr && slot_decided(vslot, I.k)) ? 1 : 0;
    // a VB2 tile none of whose parameters can change the result, from the
    // sums the prefix kernel published: skipped before anything is staged
    if (!S.skip && d == kVB2 && lam_end > lam0 &&
        vb2_tile_pruned(A, b, c, I.k, stream_len<MODE>(I), lam0, lam_end - 1,
                        flat_index(kVB2, 2, c))) {
      S.skip = 1;
      if (A.work_count != nullptr) atomicAdd(&S.wc[3], (unsigned long long)(lam_end - lam0));
    }
  }
  __syncthreads();
  if (!S.skip) node_loads<NT, MODE>(A, b, I, s_load, &S.minw, &S.err);
  __syncthreads();

  // FS1 (100 parameters) takes one parameter per thread, so that its tile
  // keeps every warp busy; the tile's parameter range (NT T G) is unchanged.
  constexpr int T_FS1 = 1;
  unsigned long long best = 0ull;
  if (!S.skip) switch (d) {
    case kMT: best = tile_dff<NT, T, kMT, MODE, false>(A, I, lam0, lam_end, s_items, s_a, s_load, S, nullptr, nullptr, -1, vslot); break;
    case kRAD2: best = tile_dff<NT, T, kRAD2, MODE, false>(A, I, lam0, lam_end, s_items, s_a, s_load, S, nullptr, nullptr, -1, vslot); break;
    case kFS1: best = tile_dff<NT, T_FS1, kFS1, MODE, false>(A, I, lam0, lam_end, s_items, s_a, s_load, S, nullptr, nullptr, -1, vslot); break;
    case kCCM1: best = tile_dff<NT, T, kCCM1, MODE, false>(A, I, lam0, lam_end, s_items, s_a, s_load, S, nullptr, nullptr, -1, vslot); break;
    case kVB2: best = tile_dff<NT, T, kVB2, MODE, false>(A, I, lam0, lam_end, s_items, s_a, s_load, S, nullptr, nullptr, -1, vslot,
                                                         A.prune && !A.verdict ? &A.keys[b] : nullptr); break;
    default: best = tile_dff<NT, T, kBJ1, MODE, false>(A, I, lam0, lam_end, s_items, s_a, s_load, S, nullptr, nullptr, -1, vslot); break;
  }
  fold_and_finalize<NT>(A, b, best, S.err != 0, ntiles, I, S.warp_key);
}

// ---------------------------------------------------------------------------
// Persistent tile loop shared by the evaluation kernels.  A kernel's tile
// table start[0..B] (nullptr: one instance with its tiles in single mode) maps
// tile t to the largest b with start[b] <= t.  Warp 0 finds it with 32-way
// probes (three dependent loads for 4096 instances instead of twelve), and
// the next tile index is fetched when the current tile starts, so that the
// atomic's latency overlaps the tile's work.
// ---------------------------------------------------------------------------
struct TileCursor {
  long long tile, inst;
};

__device__ __forceinline__ int64_t warp_find_instance(const int64_t *start, int64_t B, int64_t t) {
  int64_t lo = 0, hi = B - 1;  // invariant: start[lo] <= t
  const int lane = (int)lane_id();
  while (lo < hi) {
    const int64_t step = (hi - lo + 32) / 32;  // probes lo + j step, j < 32, cover [lo, hi]
    const int64_t idx = lo + (int64_t)lane * step;
    const bool ok = idx <= hi && start[idx] <= t;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, ok);  // bit 0 set: start[lo] <= t
    const int k = 31 - __clz((int)m);
    lo += (int64_t)k * step;
    hi = min(hi, lo + step - 1);
  }
  return lo;
}

// Publishes tile t (and its instance) to the CTA; called by every thread,
// with t taken from thread 0.
__device__ __forceinline__ void tile_publish(const int64_t *start, int64_t B, int64_t total,
                                             unsigned long long t0_value, TileCursor &cur) {
  if (threadIdx.x < 32) {
    const int64_t t = (int64_t)__shfl_sync(0xFFFFFFFFu, t0_value, 0);
    int64_t b = 0;
    if (start && t < total) b = warp_find_instance(start, B, t);
    if (threadIdx.x == 0) {
      cur.tile = t;
      cur.inst = b;
    }
  }
  __syncthreads();
}

// The first tile of this CTA: the next from the work counter, or blockIdx.x
// (also when the kernel has no tile at all: its CTAs leave without touching
// the shared counter).
__device__ __forceinline__ void tile_first(const int64_t *start, int64_t B, int64_t total,
                                           unsigned long long *work, TileCursor &cur) {
  unsigned long long t = blockIdx.x;
  if (work && threadIdx.x == 0 && total > 0) t = atomicAdd(work, 1ull);
  tile_publish(start, B, total, t, cur);
}

// Thread 0's claim on the CTA's next tile (persistent mode), issued early.
__device__ __forceinline__ unsigned long long tile_claim(unsigned long long *work) {
  return (work && threadIdx.x == 0) ? atomicAdd(work, 1ull) : ~0ull;
}

template <int MODE>
__device__ __forceinline__ InstView resolve_instance(const EvalArgs &A, int64_t b) {
  InstView I;
  I.w = nullptr;
  I.a = nullptr;
  I.begin = 0;
  if (A.tile_start == nullptr) {
    I.c = A.single_c;
    I.k = A.single_k;
    I.n = A.single_n;
    if (MODE == kSrcNodes) {
      I.w = A.base_sizes;
      I.a = A.assign;
    }
    return I;
  }
  if (MODE == kSrcNodes) {
    const int32_t base = A.node_base[b];
    I.c = A.base_capacity[base];
    I.k = A.bins[b];
    const int64_t bo = A.base_offsets[base];
    I.n = A.base_offsets[base + 1] - bo;
    I.w = A.base_sizes + bo;
    I.a = A.assign + A.assign_offsets[b];
  } else {
    I.c = A.capacity[b];
    I.k = A.bins[b];
    I.begin = A.offsets[b];
    I.n = A.offsets[b + 1] - I.begin;
  }
  return I;
}

template <int NT, int T, int G, int MODE, int MINB>
__global__ void __launch_bounds__(NT, MINB) eval_kernel(EvalArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TileShared S;
  __shared__ TileCursor cur;
  uint32_t *s_items = reinterpret_cast<uint32_t *>(smem_raw);
  float *s_a = reinterpret_cast<float *>(smem_raw + sizeof(uint32_t) * kListTop);
  uint32_t *s_load = reinterpret_cast<uint32_t *>(smem_raw + 2 * sizeof(uint32_t) * kListTop);

  pdl_wait();
  const int64_t total = A.tile_start ? A.tile_start[A.B] : A.single_tiles;
  work_count_begin(A, S);
  tile_first(A.tile_start, A.B, total, A.work, cur);
  while (cur.tile < total) {
    const int64_t t = cur.tile, b = cur.inst;
    const unsigned long long next = tile_claim(A.work);
    const int64_t t0 = A.tile_start ? A.tile_start[b] : 0;
    const int64_t nt = instance_tiles(A, b);
    const InstView I = resolve_instance<MODE>(A, b);
    process_tile<NT, T, G, MODE>(A, b, t - t0, nt, I, s_items, s_a, s_load, S);
    if (!A.work) break;
    tile_publish(A.tile_start, A.B, total, next, cur);
  }
  work_count_flush(A, S);
}

// Per-(DFF, lambda) bounds of one instance: grid (ceil(m / NT), 6); block
// (x, d) serves the requests of its index range that name DFF d.
template <int NT>
__global__ void __launch_bounds__(NT)
    debug_kernel(EvalArgs A, const int32_t *req_dff, const int64_t *req_lam, int64_t m,
                 int64_t *req_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TileShared S;
  uint32_t *s_items = reinterpret_cast<uint32_t *>(smem_raw);
  float *s_a = reinterpret_cast<float *>(smem_raw + sizeof(uint32_t) * kListTop);
  const InstView I = resolve_instance<kSrcRaggedI32>(A, 0);
  const int d = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * NT + threadIdx.x;
  int64_t idx = -1;
  if (r < m) {
    const int32_t rd = req_dff[r];
    if (d == 0 && (rd < 0 || rd >= kNumDff)) req_out[r] = -BP_ERANGE;
    if (rd == d) {
      int64_t lo, hi;
      param_range(d, I.c, lo, hi);
      const int64_t l = req_lam[r];
      if (l < lo || l > hi) req_out[r] = -BP_ERANGE;
      else idx = r;
    }
  }
  if (threadIdx.x == 0) S.err = 0;
  __syncthreads();
  switch (d) {
    case kMT: tile_dff<NT, 1, kMT, kSrcRaggedI32, true>(A, I, 0, 0, s_items, s_a, nullptr, S, req_lam, req_out, idx); break;
    case kRAD2: tile_dff<NT, 1, kRAD2, kSrcRaggedI32, true>(A, I, 0, 0, s_items, s_a, nullptr, S, req_lam, req_out, idx); break;
    case kFS1: tile_dff<NT, 1, kFS1, kSrcRaggedI32, true>(A, I, 0, 0, s_items, s_a, nullptr, S, req_lam, req_out, idx); break;
    case kCCM1: tile_dff<NT, 1, kCCM1, kSrcRaggedI32, true>(A, I, 0, 0, s_items, s_a, nullptr, S, req_lam, req_out, idx); break;
    case kVB2: tile_dff<NT, 1, kVB2, kSrcRaggedI32, true>(A, I, 0, 0, s_items, s_a, nullptr, S, req_lam, req_out, idx); break;
    default: tile_dff<NT, 1, kBJ1, kSrcRaggedI32, true>(A, I, 0, 0, s_items, s_a, nullptr, S, req_lam, req_out, idx); break;
  }
  if (S.err && idx >= 0) req_out[idx] = -BP_ERANGE;  // a size outside [0, c]
}

// ---------------------------------------------------------------------------
// vb2cap_kernel: VB2's parameter cap of Sec. 4 ("Implementation details"),
// the paper's guard against 32-bit overflow: the largest VB2 parameter is
// floor(UINT_MAX / (r max w')), r the number of items of the reduced instance
// and max w' the largest of them, and never above c (VB2's range is [2, c]);
// an instance with r = 0 or max w' = 0 keeps [2, c].  One CTA per instance
// (grid-stride); for a search node the reduced instance is its unpacked items
// (zero sizes included) and one item per non-empty bin, as in the reduction
// of Fig. 3 and its variants (transform_bins).  Writes hi[b]; an invalid
// instance (bad size or assignment, overfull bin) gets c, so that every one of
// its VB2 tiles still stages it and reports the error.  The bounds themselves
// stay exact: only the range changes.
// ---------------------------------------------------------------------------
template <int NT, int MODE>
__global__ void __launch_bounds__(NT) vb2cap_kernel(EvalArgs A, int64_t *hi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *s_load = reinterpret_cast<uint32_t *>(smem_raw);
  __shared__ int s_err;
  __shared__ uint32_t s_minw;
  __shared__ unsigned long long s_r, s_wmax;
  for (int64_t b = blockIdx.x; b < A.B; b += gridDim.x) {
    const int tid = threadIdx.x;
    if (tid == 0) {
      s_err = 0;
      s_minw = 0xFFFFFFFFu;
      s_r = 0ull;
      s_wmax = 0ull;
    }
    InstView I;
    bool ok;
    if (MODE == kSrcNodes && A.tile_start != nullptr) {
      const int32_t base = A.node_base[b];
      ok = base >= 0 && base < A.num_base;
      if (ok) ok = A.base_offsets[base + 1] - A.base_offsets[base] ==
                   A.assign_offsets[b + 1] - A.assign_offsets[b];
      if (ok) I = resolve_instance<MODE>(A, b);
      else I.c = 0;
      ok = ok && I.c >= 1 && I.c <= kMaxCapacity && I.n >= 0 && I.n <= kMaxItems && I.k >= 0 &&
           I.k <= A.max_bins &&
           (A.bin_max == nullptr || A.bin_max_offsets[b + 1] - A.bin_max_offsets[b] == I.k);
    } else {
      I = resolve_instance<MODE>(A, b);
      ok = I.c >= 1 && I.c <= kMaxCapacity && I.n >= 0 && I.n <= kMaxItems;
    }
    if (!ok) {
      if (tid == 0) hi[b] = max(I.c, (int64_t)0);
      __syncthreads();
      continue;
    }
    __syncthreads();
    uint64_t r = 0, wmax = 0;
    if (MODE == kSrcNodes) {
      for (int64_t j = tid; j < I.k; j += NT) s_load[j] = 0u;
      __syncthreads();
      for (int64_t i = tid; i < I.n; i += NT) {
        const int32_t a = I.a[i], w = I.w[i];
        if (w < 0 || (int64_t)w > I.c || a < -1 || (int64_t)a >= I.k) {
          s_err = 1;
        } else if (a >= 0) {
          const uint32_t old = atomicAdd(&s_load[a], (uint32_t)w);
          if ((int64_t)old + w > I.c) s_err = 1;
        } else {
          ++r;  // an unpacked item, zero sizes included
          wmax = max(wmax, (uint64_t)w);
          if (w > 0) atomicMin(&s_minw, (uint32_t)w);
        }
      }
      __syncthreads();
      if (!s_err && bins_transformed(A)) {
        transform_bins<NT>(A, b, I, s_load, s_minw, &s_err);
        __syncthreads();
      }
      for (int64_t j = tid; j < I.k; j += NT) {
        const uint32_t v = s_load[j];
        r += v > 0u;  // empty bins are dropped
        wmax = max(wmax, (uint64_t)v);
      }
    } else {
      if (tid == 0) r = (uint64_t)I.n;  // every entry of the list is an item
      for (int64_t q = tid; q < I.n; q += NT) {
        int64_t w = 0;
        fetch_item<MODE>(A, I, nullptr, q, w);
        if (w < 0 || w > I.c) s_err = 1;
        else wmax = max(wmax, (uint64_t)w);
      }
    }
    r = warp_sum(r);
    wmax = warp_max_u64(wmax);
    if (lane_id() == 0) {
      atomicAdd(&s_r, (unsigned long long)r);
      atomicMax(&s_wmax, (unsigned long long)wmax);
    }
    __syncthreads();
    if (tid == 0) {
      const uint64_t rw = s_r * s_wmax;  // < 2^52: r <= 2^20 + 2^14, w' <= 2^30
      int64_t v = I.c;
      // an invalid instance keeps its whole range, so that each of its VB2
      // tiles meets (and reports) the error
      if (rw != 0ull && !s_err) v = min(v, (int64_t)(4294967295ull / rw));
      hi[b] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// reduce_kernel: one CTA per node; order-preserving compaction.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT)
    reduce_kernel(EvalArgs A, const int64_t *out_offsets, int32_t *out_sizes, int64_t *out_count) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *s_load = reinterpret_cast<uint32_t *>(smem_raw);
  __shared__ int s_err;
  __shared__ int s_warp[NT / 32];
  __shared__ long long s_base;
  __shared__ uint32_t s_minw;
  for (int64_t b = blockIdx.x; b < A.B; b += gridDim.x) {
    const int tid = threadIdx.x;
    const int32_t base = A.node_base[b];
    bool ok = base >= 0 && base < A.num_base;
    const int64_t c = ok ? A.base_capacity[base] : 0;
    const int64_t bo = ok ? A.base_offsets[base] : 0;
    const int64_t n = ok ? A.base_offsets[base + 1] - bo : 0;
    const int64_t k = A.bins[b];
    ok = ok && c >= 1 && c <= kMaxCapacity && n >= 0 && n <= kMaxItems &&
         A.assign_offsets[b + 1] - A.assign_offsets[b] == n && k >= 0 && k <= A.max_bins;
    if (!ok) {
      if (tid == 0) out_count[b] = -BP_ERANGE;
      continue;
    }
    const int32_t *w = A.base_sizes + bo;
    const int32_t *a = A.assign + A.assign_offsets[b];
    if (tid == 0) {
      s_err = 0;
      s_base = 0;
      s_minw = 0xFFFFFFFFu;
    }
    for (int64_t j = tid; j < k; j += NT) s_load[j] = 0u;
    __syncthreads();
    for (int64_t i = tid; i < n; i += NT) {
      const int32_t ai = a[i], wi = w[i];
      if (wi < 0 || (int64_t)wi > c || ai < -1 || (int64_t)ai >= k) s_err = 1;
      else if (ai >= 0) {
        const uint32_t old = atomicAdd(&s_load[ai], (uint32_t)wi);
        if ((int64_t)old + wi > c) s_err = 1;
      } else if (wi > 0) {
        atomicMin(&s_minw, (uint32_t)wi);
      }
    }
    __syncthreads();
    if (bins_transformed(A) && !s_err &&
        (A.bin_max == nullptr || A.bin_max_offsets[b + 1] - A.bin_max_offsets[b] == k)) {
      InstView I;
      I.c = c;
      I.k = k;
      transform_bins<NT>(A, b, I, s_load, s_minw, &s_err);
      __syncthreads();
    } else if (A.bin_max != nullptr && A.bin_max_offsets[b + 1] - A.bin_max_offsets[b] != k) {
      s_err = 1;
      __syncthreads();
    }
    if (s_err) {
      if (tid == 0) out_count[b] = -BP_ERANGE;
      __syncthreads();
      continue;
    }
    int32_t *dst = out_sizes + out_offsets[b];
    // unpacked items, index order; then non-empty bins, bin order
    for (int64_t p = 0; p < n + k; p += NT) {
      const int64_t q = p + tid;
      bool keep = false;
      int32_t v = 0;
      if (q < n) {
        keep = a[q] == -1;
        v = w[q];
      } else if (q < n + k) {
        v = (int32_t)s_load[q - n];
        keep = v > 0;
      }
      const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
      if (lane_id() == 0) s_warp[tid >> 5] = __popc(mask);
      __syncthreads();
      int before = 0, total = 0;
      for (int e = 0; e < NT / 32; ++e) {
        before += (e < (tid >> 5)) ? s_warp[e] : 0;
        total += s_warp[e];
      }
      if (keep) dst[s_base + before + __popc(mask & ((1u << lane_id()) - 1u))] = v;
      __syncthreads();
      if (tid == 0) s_base += total;
      __syncthreads();
    }
    if (tid == 0) out_count[b] = s_base;
    __syncthreads();
  }
}

}  // namespace bplb
