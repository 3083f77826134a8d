/*
 * bp_lb.h -- C ABI of the GB300 (sm_103a) DFF lower-bound feasibility check
 * for the bin_packing constraint.
 *
 * Method: Tardivo, Michel, Pontelli, "Constraint Propagation on GPU: A Case
 * Study for the Bin Packing Constraint" (arXiv 2402.14821).
 *
 * What one check computes (Sec. 3 "Feasibility check", Sec. 3.1, Alg. 2):
 *   given the reduced instance W_R = [w'_1 .. w'_r] of a partial packing
 *   (unpacked items plus one virtual item per bin holding that bin's packed
 *   load, Fig. 3), a capacity c and a bin count k,
 *     for each DFF f in (MT, RAD2, FS1, CCM1, VB2, BJ1) and each integer
 *     parameter lambda in its range,
 *       lb(f, lambda) = ceil( sum_i f(w'_i, lambda) / f(c, lambda) )
 *     LB = max over all (f, lambda) of lb(f, lambda)
 *     the partial packing is infeasible iff LB > k.
 *   Parameter ranges (integer lambda): MT [0, c/2], RAD2 [c/4 + 1, c/3],
 *   FS1 [1, 100], CCM1 [1, c/2], VB2 [2, c], BJ1 [1, c] (integer division).
 *   The returned LB is always the full maximum (the early exit of Alg. 2 is
 *   not taken), so it does not depend on evaluation order.  The argmax is the
 *   first (f, lambda) attaining LB in the order above, lambda ascending.
 *   All arithmetic is exact integer arithmetic; results are bit-exact.
 *
 * Limits: 1 <= c <= 2^30; 0 <= every size <= c; r <= 2^20 per instance.
 *
 * Conventions
 *   - Every function returns a status code (BP_OK = 0 or a BP_E* value).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the device current when the handle was created.
 *   - The caller owns every input and output buffer.  A handle owns only its
 *     own scratch (per-instance result slots, tile tables, staging buffers).
 *   - Calls taking a `stream` (a cudaStream_t passed as void*; NULL = legacy
 *     default stream) are asynchronous and stream-ordered: outputs are valid
 *     once the stream has reached the call.  Inputs must stay valid and
 *     unchanged until then.
 *   - Per-instance domain errors found on the device (a size < 0 or > c, a
 *     capacity outside [1, 2^30], a negative bin count, a bad assignment or an
 *     overfull bin) do not fail the call: that instance's out_bound is set to
 *     -BP_ERANGE, its argmax to {-1, 0, -1} and its out_feasible to 0.
 *   - A handle is not thread-safe: calls on one handle must not overlap on
 *     the host, and asynchronous calls on one handle must be ordered on one
 *     stream (they share the handle's scratch).
 */
#ifndef BP_LB_H
#define BP_LB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BP_OK        0
#define BP_EINVAL    1  /* bad argument (NULL pointer, negative count, ...)     */
#define BP_ERANGE    2  /* a value outside the limits above                      */
#define BP_ENOMEM    3  /* a device or pinned-host allocation failed            */
#define BP_ECUDA     4  /* a CUDA runtime call failed                             */
#define BP_ETIMEOUT  5  /* a bounded wait ran out (serving layer)                 */
#define BP_EBUSY     6  /* admission refused: not enough memory budget or slots  */

/* DFF indices, in the paper's order (Alg. 2). */
#define BP_DFF_MT    0
#define BP_DFF_RAD2  1
#define BP_DFF_FS1   2
#define BP_DFF_CCM1  3
#define BP_DFF_VB2   4
#define BP_DFF_BJ1   5

typedef struct bp_lb bp_lb_t;            /* opaque handle */

/* The (DFF, lambda) pair attaining the bound: dff in 0..5, lambda its
 * integer parameter.  16 bytes, naturally aligned. */
typedef struct {
    int32_t dff;
    int32_t pad;      /* always 0 */
    int64_t lambda;
} bp_argmax_t;

/* Human-readable name of a status code (static storage). */
const char *bp_lb_strerror(int status);

/* ---- handle ---------------------------------------------------------- */

/* Creates a handle on the current CUDA device.
 *   capacity   default bin capacity c of bp_lb_eval / bp_lb_eval_node,
 *              1 <= capacity <= 2^30;
 *   max_items  largest reduced instance (and largest assignment) the plain
 *              single-check calls accept, 1 <= max_items <= 2^20; the handle
 *              allocates device and pinned staging of this size up front.
 * On success *out receives the handle.  Errors: BP_EINVAL (out NULL),
 * BP_ERANGE, BP_ENOMEM, BP_ECUDA. */
int bp_lb_create(int64_t capacity, int64_t max_items, bp_lb_t **out);

/* Releases the handle and its scratch.  Synchronises the device first.
 * NULL is accepted and ignored. */
int bp_lb_destroy(bp_lb_t *h);

/* Grows the handle's batch scratch to hold at least max_batch instances or
 * nodes, so that later batch calls with B <= max_batch allocate nothing
 * (required before capturing batch calls into a CUDA graph).
 * Errors: BP_EINVAL, BP_ENOMEM. */
int bp_lb_reserve(bp_lb_t *h, int32_t max_batch);

/* ---- plain path: one check, one launch (Alg. 3 shape) ------------------ */

/* One feasibility check of a reduced instance held in HOST memory, against
 * the handle's capacity.  Copies sizes[0..n) host->device, runs one kernel
 * launch for all six DFFs, copies the result back and synchronises (so the
 * call returns with the answer).
 *   sizes      host, n int32 item sizes of W_R, each in [0, c]; any order;
 *   n          0 <= n <= max_items (n = 0 gives LB = 0, argmax {MT, 0});
 *   bins       k >= 0;
 *   out_bound  host, receives LB;
 *   out_argmax host, receives the first attaining (DFF, lambda); may be NULL.
 * Returns BP_OK, or BP_EINVAL / BP_ERANGE (checked on the host before any
 * copy), BP_ECUDA.  The verdict is (*out_bound <= bins). */
int bp_lb_eval(bp_lb_t *h, const int32_t *sizes, int64_t n, int64_t bins,
               int64_t *out_bound, bp_argmax_t *out_argmax);

/* Plain check of one search node given as a partial packing in HOST memory:
 * base item sizes w[0..n) and assign[0..n) (-1 = unpacked, else the bin in
 * [0, bins)).  The reduction (Sec. 3, Fig. 3) runs on the device inside the
 * same single launch.  n <= max_items, bins <= max_items.  Same outputs and
 * errors as bp_lb_eval (an overfull bin gives BP_ERANGE). */
int bp_lb_eval_node(bp_lb_t *h, const int32_t *w, const int32_t *assign,
                    int64_t n, int64_t bins, int64_t *out_bound,
                    bp_argmax_t *out_argmax);

/* ---- batched path: device pointers, stream-ordered --------------------- */

/* B independent checks of reduced instances in DEVICE memory, all in one
 * stream-ordered pass (a planning launch and one persistent evaluation launch
 * over a ragged (instance, DFF, lambda-tile) grid; capturable in a CUDA graph
 * once bp_lb_reserve(h, B) has been called).
 *   B            number of instances, 0 <= B (B = 0 is a no-op);
 *   d_offsets    device int64[B+1]: instance b is d_sizes[d_offsets[b] ..
 *                d_offsets[b+1]), non-decreasing;
 *   d_sizes      device int32 sizes (bp_lb_eval_batch_i64: int64);
 *   d_capacity   device int64[B], c of each instance;
 *   d_bins       device int64[B], k of each instance;
 *   d_out_bound  device int64[B], receives LB (or -BP_ERANGE, see above);
 *   d_out_argmax device bp_argmax_t[B], may be NULL;
 *   d_out_feasible device uint8[B] (1 iff LB <= k), may be NULL;
 *   stream       cudaStream_t or NULL.
 * Errors: BP_EINVAL (NULL required pointer, B < 0), BP_ENOMEM, BP_ECUDA. */
int bp_lb_eval_batch(bp_lb_t *h, int32_t B, const int64_t *d_offsets,
                     const int32_t *d_sizes, const int64_t *d_capacity,
                     const int64_t *d_bins, int64_t *d_out_bound,
                     bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                     void *stream);

int bp_lb_eval_batch_i64(bp_lb_t *h, int32_t B, const int64_t *d_offsets,
                         const int64_t *d_sizes, const int64_t *d_capacity,
                         const int64_t *d_bins, int64_t *d_out_bound,
                         bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                         void *stream);

/* B search nodes in DEVICE memory: each node is a partial packing of one of
 * the base instances; its reduced instance (Sec. 3 "Feasibility check",
 * Fig. 3: unpacked items plus one virtual item of size equal to the packed
 * load per non-empty bin) is built on the device inside the evaluation launch
 * and checked as in bp_lb_eval_batch.
 *   num_base         I, the number of base instances;
 *   d_base_offsets   device int64[I+1] ragged offsets of the base instances;
 *   d_base_sizes     device int32 base item sizes;
 *   d_base_capacity  device int64[I], c of each base instance;
 *   d_node_base      device int32[B], base instance of each node (0..I-1);
 *   d_assign_offsets device int64[B+1]: node b's assignment is
 *                    d_assign[d_assign_offsets[b] ..) with exactly n = size of
 *                    its base instance entries;
 *   d_assign         device int32: -1 unpacked, else bin index in [0, bins);
 *   d_bins           device int64[B], k of each node, 0 <= k <= max_bins;
 *   max_bins         host bound on every d_bins[b], 0 <= max_bins <= 16384
 *                    (sizes the on-chip load table; BP_ERANGE above it);
 *   outputs as for bp_lb_eval_batch.
 * A node with an out-of-range bin index or an overfull bin gets the
 * per-instance error described above. */
int bp_lb_eval_nodes(bp_lb_t *h, int32_t B, int32_t num_base,
                     const int64_t *d_base_offsets,
                     const int32_t *d_base_sizes, const int64_t *d_base_capacity,
                     const int32_t *d_node_base, const int64_t *d_assign_offsets,
                     const int32_t *d_assign, const int64_t *d_bins,
                     int64_t max_bins, int64_t *d_out_bound,
                     bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                     void *stream);

/* The reduction alone (Sec. 3 "Feasibility check", Fig. 3), for B nodes laid
 * out as in bp_lb_eval_nodes.  Node b's reduced instance is written to
 * d_out_sizes[d_out_offsets[b] ..) -- the caller reserves n + bins entries
 * there -- as the unpacked items in index order followed by the loads of the
 * non-empty bins in bin order; d_out_count[b] receives its length r, or
 * -BP_ERANGE for a node with a bad assignment or an overfull bin.
 * Errors: BP_EINVAL, BP_ERANGE (max_bins), BP_ECUDA. */
int bp_lb_reduce_nodes(bp_lb_t *h, int32_t B, int32_t num_base,
                       const int64_t *d_base_offsets,
                       const int32_t *d_base_sizes,
                       const int64_t *d_base_capacity,
                       const int32_t *d_node_base,
                       const int64_t *d_assign_offsets,
                       const int32_t *d_assign, const int64_t *d_bins,
                       int64_t max_bins, const int64_t *d_out_offsets,
                       int32_t *d_out_sizes, int64_t *d_out_count,
                       void *stream);

/* ---- batched path without a handle and without allocation ---------------- */

/* Largest B bp_lb_eval_batch_noalloc accepts. */
#define BP_NOALLOC_MAX_BATCH 4096

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory where they check: code whose device
 * memory belongs to another allocator (e.g. a framework pool that reserved
 * the whole device), search loops that must not take the device-wide
 * synchronisation of cudaFree between their own kernels, and solvers with a
 * device-memory budget fixed at start-up.  It computes exactly what
 * bp_lb_eval_batch computes, with the same arguments and per-instance error
 * convention, but needs no handle and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   Its scratch (tile table, result slots, counters: about 82 KB) is one
 *   fixed __device__ array in the library, held by every GPU that loads the
 *   library until the process exits.
 *   The first call on a device (B = 0 is allowed, as a warm-up with NULL
 *   pointers) does a one-time set-up with the device current: it looks up
 *   that array's device address (cudaGetSymbolAddress) and queries the two
 *   kernels it launches.  Under CUDA's lazy module loading (the default,
 *   CUDA_MODULE_LOADING=LAZY) that is when the driver loads this library's
 *   kernels and the array onto the device, which may take device memory, so
 *   make that first call at start-up, before another allocator takes the
 *   device and before any stream capture on it.  The address is kept per
 *   device for the life of the process: cudaDeviceReset after the first
 *   call is not supported.
 *   All calls share the one array: calls whose work overlaps on the GPU (on
 *   different streams, or from different host threads) race and give wrong
 *   results; order them on one stream.  Each call clears the parts it uses.
 *   It evaluates every DFF item by item in the generic kernel (the
 *   BP_ALGO_DIRECT algorithm, VB2 included) with launch shape 0 and no
 *   autotuning: the prefix-count tables and the separate VB2 kernel need
 *   scratch that only a handle owns.  At large capacities that costs several
 *   times a handle's default path, more as c grows.
 * Errors: BP_EINVAL (NULL required pointer, B < 0), BP_ERANGE
 * (B > BP_NOALLOC_MAX_BATCH, checked before any launch), BP_ECUDA. */
int bp_lb_eval_batch_noalloc(int32_t B, const int64_t *d_offsets,
                             const int32_t *d_sizes, const int64_t *d_capacity,
                             const int64_t *d_bins, int64_t *d_out_bound,
                             bp_argmax_t *d_out_argmax,
                             uint8_t *d_out_feasible, void *stream);

/* ---- evaluation algorithm ------------------------------------------------ */

/* BP_ALGO_DIRECT evaluates every (DFF, lambda) pair item by item (Alg. 2's
 * loops).  BP_ALGO_PREFIX (the default) computes the same bounds exactly but
 * evaluates MT, RAD2, FS1, CCM1 and BJ1 from value-indexed suffix counts and
 * sums of the reduced instance (O(1), O(1), O(lambda), O(c / lambda) and
 * O(c / lambda) lookups per parameter instead of one evaluation per item)
 * when the reduced sizes sum to less than 2^31.  The tables live in one
 * CTA's shared memory where they fit in 48 KB (c up to 12286 for RAD2, FS1,
 * BJ1 and the merged MT/RAD2/CCM1 tile, 24574 for MT and CCM1 alone); else,
 * with cluster tables on (bp_lb_set_cluster_tables), spread over
 * the shared memory of a cluster of 8 CTAs, 64 KB each (c up to 131070, MT
 * and CCM1 alone 262142); else in a global-memory scratch of 4 MB per CTA
 * (c up to 1048574, MT and CCM1 alone 2097150); beyond that on the direct
 * path.  VB2 stays on the direct kernels, except that in batched calls with
 * pruning on (or in verdict mode) the merged MT/RAD2/CCM1 tile also takes
 * VB2 when pruning leaves only parameters up to some lmax and their
 * count-table lookups (about l / 2 each) stay within 65536 per CTA of the
 * tile.  Results are identical either way. */
#define BP_ALGO_DIRECT 0
#define BP_ALGO_PREFIX 1

/* Selects the algorithm of a handle.  Errors: BP_EINVAL, BP_ERANGE. */
int bp_lb_set_algorithm(bp_lb_t *h, int32_t algo);

/* Cluster tables on (1) or off (0, the default): with them on, prefix-count
 * tables too large for one CTA's 48 KB but within 512 KB are built and read
 * by a cluster of 8 CTAs in their shared memory (one launch more per batched
 * call, the cluster kernel, which finds nothing to do when no instance has
 * such tables); off, they go to the global scratch as beyond 512 KB.  A
 * cluster takes one such instance's tables several times faster than one CTA
 * with its tables in the global scratch, but occupies eight CTAs, so it pays
 * for batches with fewer such instances than the GPU has CTA slots; the
 * batched autotuners (bp_lb_autotune_batch, bp_lb_autotune_nodes) try both
 * settings.  The paper has no counterpart (its kernel evaluates every pair
 * item by item); results are identical either way.  Errors: BP_EINVAL (NULL handle), BP_ERANGE (not 0
 * or 1).  bp_lb_get_cluster_tables: the setting, or -1 for a NULL handle. */
int bp_lb_set_cluster_tables(bp_lb_t *h, int32_t on);
int bp_lb_get_cluster_tables(bp_lb_t *h);

/* The handle's algorithm (batched modes), or -1 for a NULL handle. */
int bp_lb_get_algorithm(bp_lb_t *h);

/* ---- result mode: full maximum or verdict only ---------------------------- */

/* BP_RESULT_FULL (the default) returns, per instance, the exact maximum over
 * every (DFF, lambda) bound and its first argmax (reading R3 of the design:
 * Alg. 2 without its early exit), and the verdict bound <= k.
 * BP_RESULT_VERDICT returns the verdict only, exactly, with Alg. 2's early
 * exit (Sec. 3.1, Alg. 2): once any bound of an instance exceeds k, its
 * remaining tiles stop (a flag -- the instance's result slot -- read by every
 * kernel when it starts a tile and between parameter groups), and on the VB2
 * path a parameter is skipped when an upper bound on its bound, from the
 * instance's sums alone, is <= k (it cannot change the verdict; this holds
 * with VB2 pruning off too).  The cheap DFFs run first (the prefix-count kernel,
 * then VB2, then the rest), so a decided instance skips the expensive ones.
 * In this mode out_feasible is exact; out_bound / out_argmax hold a genuine
 * bound of the instance and the (DFF, lambda) that gives it: one above k
 * when infeasible (which one may vary between runs), one <= k when feasible
 * (the largest evaluated, not necessarily the maximum).
 * Errors: BP_EINVAL (NULL handle), BP_ERANGE (unknown mode). */
#define BP_RESULT_FULL 0
#define BP_RESULT_VERDICT 1
int bp_lb_set_result_mode(bp_lb_t *h, int32_t mode);

/* The handle's result mode, or -1 for a NULL handle. */
int bp_lb_get_result_mode(bp_lb_t *h);

/* ---- reduction variants (search-node mode) --------------------------------- */

/* The paper's reduction (Sec. 3 "Feasibility check", Fig. 3) turns each
 * non-empty bin of a search node into one item of its packed load
 * (BP_REDUCE_LOADS, the default).  Two variants, not defined in the paper
 * (they keep every bound valid: any completion of the partial packing still
 * fits the reduced instance in the k bins):
 *   BP_REDUCE_CLOSE  a bin whose free space is smaller than every unpacked
 *                    item of nonzero size (every bin, when there is none)
 *                    can take nothing more: its item is c;
 *   bin maximum loads (bp_lb_set_bin_max): a bin that may hold at most
 *                    cap_j <= c becomes an item of load + c - cap_j (the
 *                    capacity it cannot use is filled), then CLOSE applies
 *                    to that item when set.
 * The mode applies to every search-node call of the handle
 * (bp_lb_eval_nodes, bp_lb_eval_node, bp_lb_reduce_nodes); the maximum loads
 * to the batched ones (bp_lb_eval_nodes, bp_lb_reduce_nodes).
 * Errors: BP_EINVAL (NULL handle), BP_ERANGE (unknown mode). */
#define BP_REDUCE_LOADS 0
#define BP_REDUCE_CLOSE 1
int bp_lb_set_reduction(bp_lb_t *h, int32_t mode);

/* The handle's reduction mode, or -1 for a NULL handle. */
int bp_lb_get_reduction(bp_lb_t *h);

/* Per-bin maximum loads for the handle's batched search-node calls: node b's
 * bin j may hold at most d_bin_max[d_offsets[b] + j], which must lie in
 * [0, c] and be at least the bin's packed load (else that node's result is
 * -BP_ERANGE); d_offsets[b + 1] - d_offsets[b] must equal the node's bins.
 * Device pointers owned by the caller, read by every later batched
 * search-node call until cleared (both NULL).  Errors: BP_EINVAL (NULL
 * handle, or exactly one pointer NULL). */
int bp_lb_set_bin_max(bp_lb_t *h, const int64_t *d_offsets, const int32_t *d_bin_max);

/* ---- VB2 pruning ------------------------------------------------------------ */

/* On (1, the default): in both result modes a VB2 parameter is skipped when
 * an upper bound on its bound, from the instance's sums alone (sum of
 * ceil(x) < sum of (x + 1) over the small items, >= x over the big ones),
 * shows it cannot change the result: in full mode when that upper bound is
 * below the instance's best bound so far -- or equal to it, with the best one
 * earlier in (DFF, lambda) order -- read from the instance's result slot
 * (it only grows, and the prefix-count kernel has filled it before VB2
 * runs); in verdict mode when it is <= k.  Results are identical with
 * pruning off (0); only the work differs.  Errors: BP_EINVAL (NULL handle),
 * BP_ERANGE (not 0 or 1). */
int bp_lb_set_pruning(bp_lb_t *h, int32_t on);

/* The handle's pruning switch, or -1 for a NULL handle. */
int bp_lb_get_pruning(bp_lb_t *h);

/* ---- VB2's parameter cap (the paper's overflow guard) ----------------------- */

/* Sec. 4 ("Implementation details") limits VB2's parameter to
 * floor(UINT_MAX / (r max w')), UINT_MAX = 2^32 - 1, r the number of items of
 * the reduced instance and max w' the largest of them, because the paper's
 * kernels hold VB2's intermediates in unsigned 32-bit integers.  This library
 * computes every bound exactly and by default evaluates VB2 over its whole
 * printed range [2, c] (Sec. 3.1).  With the cap on (1), VB2 is evaluated over
 * [2, min(c, floor(UINT_MAX / (r max w')))] instead (the whole range when
 * r max w' = 0; no VB2 parameter at all when the floor is below 2), so that
 * the bound the paper's implementation computes can be reproduced; the other
 * DFFs and the arithmetic are unchanged.  r counts every entry of a reduced
 * instance given as a list (zero sizes included) and, for a search node, its
 * unpacked items plus one item per non-empty bin (after a reduction variant,
 * per bp_lb_set_reduction).  Applies to every evaluation call of the handle
 * (batched and plain; not bp_lb_debug_params, which takes any lambda in
 * [2, c]); costs one extra launch per call.  An invalid instance is reported
 * as without the cap.  Default off (0).
 * Errors: BP_EINVAL (NULL handle), BP_ERANGE (not 0 or 1). */
int bp_lb_set_vb2_cap(bp_lb_t *h, int32_t on);

/* The handle's VB2 cap switch, or -1 for a NULL handle. */
int bp_lb_get_vb2_cap(bp_lb_t *h);

/* ---- L2, the comparator ---------------------------------------------------- */

/* Martello and Toth's L2 (Sec. 3.1, the bound the DFF collection replaces)
 * of B ragged instances, on the device: L2 = max over integer lambda in
 * [0, floor(c/2)] of |W1| + |W2| + max(0, ceil((sum W3 - (c |W2| - sum W2)) / c)).
 * One CTA per instance sorts its items in shared memory and evaluates every
 * lambda where the sets change (O(r log r)); results are exact.
 *   d_offsets   device int64[B+1], instance b is d_sizes[d_offsets[b] .. d_offsets[b+1]);
 *   d_sizes     device int32, each in [0, c];
 *   d_capacity  device int64[B], 1 <= c <= 2^30;
 *   d_out_l2    device int64[B] (caller-owned): L2, or -BP_ERANGE for an
 *               instance with a size outside [0, c], a bad capacity or more
 *               than 8192 items;
 *   stream      a cudaStream_t (NULL: the legacy default stream).
 * Stream-ordered; returns BP_EINVAL for NULL pointers or B < 0. */
int bp_lb_l2_batch(bp_lb_t *h, int32_t B, const int64_t *d_offsets, const int32_t *d_sizes,
                   const int64_t *d_capacity, int64_t *d_out_l2, void *stream);

/* ---- which DFFs make up the bound ----------------------------------------- */

/* Bit d of `mask` keeps DFF d (BP_DFF_MT = 0 ... BP_DFF_BJ1 = 5) in the
 * bound; the default is all six (63).  With a single DFF f the result is its
 * own bound L_f = max over lambda of ceil(sum f(w, lambda) / f(c, lambda))
 * and its first argmax (Sec. 3.1, Table 1 reports these per DFF).  When
 * every DFF left in has an empty parameter range at an instance's capacity
 * (RAD2 at c in {1, 2, 4, 5, 8}, VB2 and CCM1 at c = 1), that instance's
 * bound is 0 with argmax {-1, 0, -1} (the plain path then returns without a
 * launch and without checking a node's assignment).  Applies to every call
 * of the handle.  Errors: BP_EINVAL (NULL handle), BP_ERANGE (mask outside
 * 1..63). */
int bp_lb_set_dff_mask(bp_lb_t *h, int32_t mask);

/* The handle's DFF mask, or -1 for a NULL handle. */
int bp_lb_get_dff_mask(bp_lb_t *h);

/* ---- concurrency of the evaluation kernels (batched calls) ----------------- */

/* A batched call runs four evaluation kernels (see bp_lb_kernel_times4), by
 * default (0) one after another on the caller's stream.  With
 * prefix_ctas_per_sm > 0 the cluster and prefix-count kernels, then the
 * generic kernel, run on a high-priority side stream of the handle while the
 * VB2 kernel runs
 * on the caller's stream: the prefix kernel takes that many CTAs per SM, the
 * VB2 kernel the rest (its remaining CTAs become resident as the prefix
 * kernel's retire).  The call stays ordered on the caller's stream (fork
 * after the planning kernel, join before the call's work is complete) and can
 * be captured in a CUDA graph.  Results are identical either way; on the
 * search-node batch the serial order is the faster one.
 * Errors: BP_EINVAL (NULL handle), BP_ERANGE (outside 0..8). */
int bp_lb_set_overlap(bp_lb_t *h, int32_t prefix_ctas_per_sm);

/* Measurement aid: with timing on, every batched call records CUDA events
 * on their streams around its three evaluation launches -- the prefix-count
 * kernel, the VB2 kernel (VB2 at c <= 65535, evaluated item by item with its
 * fixed-point quotients) and the generic direct kernel (every other (DFF,
 * lambda) evaluated item by item) -- (not for use under stream capture).
 * bp_lb_kernel_times waits for the events recorded since the previous query
 * and returns the total milliseconds of each kernel and the number of calls
 * (any pointer may be NULL).  bp_lb_kernel_times4 does the same with the
 * cluster kernel's time too: out_ms4 = {cluster, prefix, VB2, direct} (NULL:
 * not written); either query consumes the events. */
int bp_lb_set_kernel_timing(bp_lb_t *h, int32_t on);
int bp_lb_kernel_times(bp_lb_t *h, double *ms_prefix, double *ms_vb2, double *ms_direct,
                       int64_t *calls);
int bp_lb_kernel_times4(bp_lb_t *h, double *out_ms4, int64_t *calls);

/* Measurement aid: work counted by the batched calls made with timing on,
 * since the previous query (which resets the counters; it synchronizes the
 * device): out4[0] VB2 (item, parameter) pairs evaluated by the VB2 kernel,
 * out4[1] VB2 pairs evaluated by the generic kernel, out4[2] VB2 parameters
 * evaluated, out4[3] VB2 parameters pruned (bp_lb_set_pruning).
 * Errors: BP_EINVAL (NULL pointer), BP_ECUDA. */
int bp_lb_kernel_work(bp_lb_t *h, int64_t *out4);

/* Measurement aid with no counterpart in the paper: the integer instruction
 * issue rate of the current device, the peak against which the item-by-item
 * kernels' roofline is reported.  Launches (stream-ordered, asynchronous)
 * blocks_per_sm x SM-count CTAs of 256 threads that run only integer
 * multiply-adds and xors in eight independent chains per thread (the two
 * half-rate integer pipes together allow one warp instruction per clock per
 * sub-partition), `trips` loop trips of 256 such operations each, and writes
 * one word per thread to d_sink (device, caller-owned, at least
 * blocks_per_sm x SM-count x 256 uint32).  *out_lane_ops receives the
 * number of integer lane operations the launch performs; divided by the
 * launch's CUDA-event time it is the sustained integer issue rate.
 * Errors: BP_EINVAL (blocks_per_sm outside 1..8, trips < 1, NULL pointer),
 * BP_ECUDA. */
int bp_lb_probe_int_issue(int32_t blocks_per_sm, int32_t trips, uint32_t *d_sink,
                          void *stream, int64_t *out_lane_ops);

/* ---- launch shapes and autotuning ---------------------------------------- */

/* Input modes of the evaluation kernel, for the launch-shape calls below. */
#define BP_MODE_RAGGED_I32 0   /* bp_lb_eval, bp_lb_eval_batch     */
#define BP_MODE_RAGGED_I64 1   /* bp_lb_eval_batch_i64             */
#define BP_MODE_NODES      2   /* bp_lb_eval_nodes                 */
#define BP_MODE_PLAIN_RAGGED 3 /* bp_lb_eval (plain path)          */
#define BP_MODE_PLAIN_NODES  4 /* bp_lb_eval_node (plain path)     */

/* The evaluation kernel is compiled for a small table of launch shapes:
 * nt threads per CTA, t parameters per thread and pass, g passes per tile
 * (so a tile covers nt*t*g consecutive parameters of one DFF), and a floor of
 * min_blocks resident CTAs per SM (which caps registers per thread).  This is
 * the implementation's own tuning space; the paper uses one parameter per
 * thread and blocks of one SM's core count (Sec. 4, "Parallelization"). */
int bp_lb_num_launch_shapes(void);

/* Describes shape `id` (0 <= id < bp_lb_num_launch_shapes()); any output
 * pointer may be NULL.  Errors: BP_ERANGE. */
int bp_lb_launch_shape_info(int32_t id, int32_t *nt, int32_t *t, int32_t *g,
                            int32_t *min_blocks);

/* Selects the shape the handle uses for one mode (default 0 for the batched
 * modes; a short-tile latency shape for the plain modes, which spread one
 * check over all SMs).
 * Errors: BP_EINVAL (bad handle or mode), BP_ERANGE (bad id). */
int bp_lb_set_launch_shape(bp_lb_t *h, int32_t mode, int32_t id);

/* The shape the handle uses for `mode`, or -1 for a bad handle or mode. */
int bp_lb_get_launch_shape(bp_lb_t *h, int32_t mode);

/* Autotuner: runs the given batch once per launch shape to warm up, then
 * `reps` times, timed with CUDA events on `stream`; keeps the fastest shape
 * for the mode and writes it to *best_shape (may be NULL), and the mean
 * milliseconds per call of every shape to ms_per_shape[0 .. num shapes) (may
 * be NULL); then times the batch with that shape and cluster tables switched
 * (bp_lb_set_cluster_tables) and keeps the setting 3% faster or more, never
 * leaving them on for a batch with no instance whose tables are of their size.  The output buffers receive the batch's results.  Synchronises
 * the stream (not capturable).  Arguments as for bp_lb_eval_batch(_i64)
 * (sizes_are_i64 selects the size type) and bp_lb_eval_nodes.
 * Errors: as those calls, and BP_EINVAL for B < 1 or reps < 1. */
int bp_lb_autotune_batch(bp_lb_t *h, int32_t B, const int64_t *d_offsets,
                         const void *d_sizes, int32_t sizes_are_i64,
                         const int64_t *d_capacity, const int64_t *d_bins,
                         int64_t *d_out_bound, bp_argmax_t *d_out_argmax,
                         uint8_t *d_out_feasible, int32_t reps,
                         float *ms_per_shape, int32_t *best_shape,
                         void *stream);

int bp_lb_autotune_nodes(bp_lb_t *h, int32_t B, int32_t num_base,
                         const int64_t *d_base_offsets,
                         const int32_t *d_base_sizes,
                         const int64_t *d_base_capacity,
                         const int32_t *d_node_base,
                         const int64_t *d_assign_offsets,
                         const int32_t *d_assign, const int64_t *d_bins,
                         int64_t max_bins, int64_t *d_out_bound,
                         bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                         int32_t reps, float *ms_per_shape,
                         int32_t *best_shape, void *stream);

/* Plain-path autotuner: times `reps` bp_lb_eval_node calls (host wall
 * clock; each call synchronises) with every algorithm and launch shape on the
 * given node and keeps the fastest for the plain node path.  us_per_shape
 * (may be NULL) receives 2 * bp_lb_num_launch_shapes() values: first every
 * shape with BP_ALGO_DIRECT, then every shape with BP_ALGO_PREFIX;
 * *best_shape (may be NULL) the winning index into that list.
 * Errors: as bp_lb_eval_node, BP_EINVAL for reps < 1. */
int bp_lb_autotune_plain_node(bp_lb_t *h, const int32_t *w, const int32_t *assign,
                              int64_t n, int64_t bins, int32_t reps,
                              float *us_per_shape, int32_t *best_shape);

/* ---- serving: continuous batching of checks from concurrent searches ---- */

/* A request loop for many concurrent searches (the paper's CP solver issues
 * one check per propagation of the bin_packing constraint, Alg. 1).  Base
 * instances are registered once and stay resident on the device; a check is
 * a partial packing of one of them.  A scheduler thread forms batches from
 * pending checks whenever one of `slots` in-flight slots frees up and runs
 * them with bp_lb_eval_nodes on that slot's own stream and scratch, so a
 * batch admitted while others run shares the SMs with them.  Admission is by
 * device-memory footprint: the resident pool holds at most pool_items sizes
 * and at most max_queued_items assignment entries may be pending or in
 * flight; a request that does not fit is refused with BP_EBUSY and should be
 * retried after polling.  Results are identical to bp_lb_eval_nodes on the
 * same node (every check is independent of the others in its batch). */
typedef struct bp_serve bp_serve_t;

typedef struct {
    int64_t request;      /* id returned by bp_serve_submit                     */
    int64_t tag;          /* the caller's tag                                    */
    int64_t bound;        /* LB, or -BP_ERANGE (bad node) / -BP_ECUDA             */
    bp_argmax_t argmax;   /* first attaining (DFF, lambda)                       */
    double latency_us;    /* from submit to the result being collected           */
    int32_t status;       /* BP_OK, BP_ERANGE or BP_ECUDA                         */
    uint8_t feasible;     /* 1 iff bound <= bins                                  */
    uint8_t pad[3];
} bp_serve_result_t;

/* Creates a server on the current device and starts its scheduler thread.
 *   pool_items        device slots for resident base-instance sizes (int32);
 *   max_instances     most instances that can be registered;
 *   max_queued_items  bound on the assignment entries of pending plus
 *                     in-flight checks (each slot stages max_queued_items /
 *                     slots of them, which also bounds one instance's size);
 *   slots             batches in flight at once, 1..16;
 *   max_batch         checks per batch;
 *   max_bins          bound on any check's bin count (<= 16384).
 * Errors: BP_EINVAL, BP_ERANGE, BP_ENOMEM, BP_ECUDA. */
int bp_serve_create(int64_t pool_items, int32_t max_instances,
                    int64_t max_queued_items, int32_t slots, int32_t max_batch,
                    int64_t max_bins, bp_serve_t **out);

/* Finishes every pending and in-flight check, stops the scheduler and frees
 * the server.  Results not yet polled are discarded. */
int bp_serve_destroy(bp_serve_t *s);

/* Uploads a base instance (host sizes, each in [0, capacity]) to the
 * resident pool; *out_id receives its id.  BP_EBUSY when the pool or the
 * instance table is full; BP_ERANGE for bad sizes, capacity or an instance
 * larger than a slot. */
int bp_serve_register(bp_serve_t *s, const int32_t *sizes, int64_t n,
                      int64_t capacity, int32_t *out_id);

/* Queues one check of a registered instance: assign[0..n) host (n = the
 * instance's size; -1 = unpacked, else a bin in [0, bins)); the array is
 * copied before the call returns.  *out_request (may be NULL) receives the
 * request id.  BP_EBUSY when the queued-entries bound would be exceeded;
 * BP_EINVAL for an unknown instance; BP_ERANGE for bins outside
 * [0, max_bins].  A bad assignment or overfull bin is reported in the
 * result (status BP_ERANGE). */
int bp_serve_submit(bp_serve_t *s, int32_t instance, const int32_t *assign,
                    int64_t bins, int64_t tag, int64_t *out_request);

/* Moves up to max_results finished checks to out[] and their number to
 * *count, waiting up to wait_us microseconds for the first one (0 = do not
 * wait).  Returns BP_ETIMEOUT when it waited and nothing finished. */
int bp_serve_poll(bp_serve_t *s, bp_serve_result_t *out, int32_t max_results,
                  int32_t *count, int32_t wait_us);

/* Counters (any pointer may be NULL).  Returns the scheduler's status:
 * BP_OK, or BP_ECUDA once a batch failed on the device. */
int bp_serve_stats(bp_serve_t *s, int64_t *pending, int64_t *queued_items,
                   int64_t *batches, int64_t *done, int64_t *refused);

/* ---- one instance over a range of parameters (sharding one check) -------- */

/* The bound of Alg. 2 restricted to a contiguous range of parameters: the
 * flattened index g numbers every (DFF, lambda) pair in the paper's order
 * (MT, RAD2, FS1, CCM1, VB2, BJ1; lambda ascending within a DFF; Sec. 3.1
 * ranges), 0 <= g < P(c) = sum of bp_lb_param_count over the six DFFs.  Over
 * the pairs with g0 <= g < g1 this computes the largest bound and the
 * smallest g attaining it, packed into one key
 *   key = (bound << 32) | (2^32 - 1 - g),
 * so that the maximum key over a partition of [0, P(c)) into ranges is the
 * full bound and its first argmax (the collection's maximum, Alg. 2, with the
 * first-attaining tie-break): one instance too large for one GPU is split
 * over ranks by range, and the ranks' keys meet in one 8-byte MAX all-reduce.
 *   d_sizes   device int32 sizes of the reduced instance, n of them, each in
 *             [0, c];
 *   c         its capacity, 1 <= c <= 2^30;
 *   g0, g1    0 <= g0 <= g1 <= P(c);
 *   d_out_key device int64[1] (caller-owned): the key; 0 when the range holds
 *             no parameter (of the handle's DFF mask); -BP_ERANGE for a size
 *             outside [0, c] (found by the range's evaluation).
 * Every pair is evaluated item by item in the generic kernel (the handle's
 * launch shape for BP_MODE_RAGGED_I32); the handle's DFF mask, VB2 pruning
 * (exact, against the range's own best key) and VB2 cap apply.  Stream-
 * ordered on `stream`; calls on one handle must be ordered on one stream.
 * Errors: BP_EINVAL (NULL handle or pointer, n < 0), BP_ERANGE (c, n, or the
 * range outside the limits above), BP_ECUDA. */
int bp_lb_eval_range(bp_lb_t *h, const int32_t *d_sizes, int64_t n,
                     int64_t c, int64_t g0, int64_t g1, int64_t *d_out_key,
                     void *stream);

/* ---- inspection -------------------------------------------------------- */

/* Per-parameter bounds for spot checks of very long sweeps: for j < m,
 * d_out_lb[j] = lb(d_dff[j], d_lambda[j]) of the single reduced instance
 * d_sizes[0..n) with capacity c, computed by the same device code as the
 * batched path (one lambda per lane).  A lambda outside its DFF's range
 * gives -BP_ERANGE.  Device pointers; stream-ordered. */
int bp_lb_debug_params(bp_lb_t *h, const int32_t *d_sizes, int64_t n,
                       int64_t c, const int32_t *d_dff,
                       const int64_t *d_lambda, int64_t m, int64_t *d_out_lb,
                       void *stream);

/* Number of integer parameters of DFF d at capacity c (0 for an empty
 * range), and the range itself; host-only helper, no device work.
 * Returns -1 for a bad d or c. */
int64_t bp_lb_param_count(int32_t d, int64_t c, int64_t *lo, int64_t *hi);

/* Which path evaluates DFF d of an instance with capacity c whose item
 * stream has stream_len entries (reduced items, or base items plus bins for a
 * search node) under algorithm `algo`: BP_ALGO_PREFIX or BP_ALGO_DIRECT;
 * -1 for bad arguments.  Host-only, for accounting. */
int bp_lb_dff_route(int32_t d, int64_t c, int64_t stream_len, int32_t algo);

/* Host-side exhaustive self-check of the exact division used by the kernels
 * (Granlund-Montgomery multiply-high division by invariant integers):
 * compares it with '/' for every divisor in [d_lo, d_hi] on every numerator
 * in [0, n_hi] and on `samples` pseudo-random numerators in [0, 2^31).
 * Returns the number of mismatches (0 expected), -1 on bad arguments. */
int64_t bp_lb_selfcheck_division(uint32_t d_lo, uint32_t d_hi, uint32_t n_hi,
                                 int64_t samples);

#ifdef __cplusplus
}
#endif

#endif /* BP_LB_H */
