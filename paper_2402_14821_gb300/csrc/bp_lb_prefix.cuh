// bp_lb_prefix.cuh -- prefix-count evaluation of MT, RAD2, FS1, CCM1 and BJ1.
//
// Same bounds as the direct evaluators (bit-exact), asymptotically less work:
// per tile the instance's items are histogrammed by value in shared memory and
// suffix-scanned, after which each parameter needs O(1) (MT, RAD2), O(l)
// (FS1), O(U / l) (CCM1) or O(c / l) (BJ1) table lookups instead of one
// evaluation per item.
// With u, the small/big classes and cm = c mod l as in bp_lb_core.cuh, and the
// u-domain tables (x in [0, U + 1], U = floor((c - 1) / 2), entry U + 1 = 0)
//   E(x)  = sum_small u [u >= x] - sum_big u [u >= x],
//   N'(x) = #small[u >= x] - #big[u >= x],   Ns(x) = #small[u >= x],
// and the w-domain table (x in [0, c + 1]) NN(x) = sum_w max(0, w - x + 1):
//   MT:   sum_small u [u >= l] + sum_big u [u < l] = E(l) + TB, TB = sum_big u;
//   RAD2: #small[u >= l] - #big[u >= l] = N'(l), and with y = c - 2l + 1
//         #small[u > c - 2l] = Ns(y), #big[u > c - 2l] = Ns(y) - N'(y);
//   CCM1: sum_small floor(u / l) - sum_big floor(u / l) = sum_{j >= 1} N'(j l),
//         since floor(u / l) counts the multiples j l <= u;
//   BJ1:  cm q + min(rho, cm) (w = q l + rho) counts the x <= w in the union
//         of the blocks [j l + 1, j l + cm], j >= 0, so summed over the items
//         it is sum_j (NN(j l + 1) - NN(j l + cm + 1)) over j = 0 .. floor(c / l),
//         and S = sum w minus that.  With q = floor(c / l), j l + cm + 1 =
//         c + 1 - (q - j) l, NN(1) = sum w and NN(c + 1) = 0, the terms pair up
//         into S = sum_{i=1}^{q} D(i l), D(x) = NN(c + 1 - x) - NN(1 + x): one
//         lookup per multiple of l, like CCM1.  D overwrites NN in place (the
//         pair x, c - x reads and writes the same two entries) once FS1 is done;
//   FS1:  with l' = l + 1, w maps to w l when c divides w l', else to
//         floor(w l' / c) c, so S = c sum_w floor(w l' / c) - sum_{c | w l'} w;
//         floor(w l' / c) counts the j in [1, l'] with w >= ceil(j c / l'), and
//         c divides w l' exactly for the multiples w = m c / gcd(c, l'):
//         S = c sum_{j=1}^{l'} N(ceil(j c / l')) - sum_m m g #[w = m g].
// NN is the suffix sum of the suffix count N(x) = #[w >= x]: a histogram
// scanned twice; N(x) = NN(x) - NN(x + 1), #[w = x] = N(x) - N(x + 1).  Every
// table entry and every sum above is bounded by the instance's size total,
// below 2^31 on this path (prefix_handles), so the tables and accumulators are
// 32-bit (FS1's S, up to l' times the total, is formed in 64 bits).  VB2 stays
// on the direct kernels.
//
// Only bounds above L1 = ceil(sum w / c) can change the maximum: L1 is MT's
// bound at l = 0, the smallest flattened index, which wins every tie at L1.
// Each thread keeps its best bound B (starting at L1) and only divides for a
// parameter whose sum S exceeds B f(c, l), i.e. whose bound exceeds B; since a
// thread meets its parameters in increasing order, an equal bound later never
// displaces the earlier one, exactly as in the full maximum.
#pragma once

#include "bp_lb_kernels.cuh"

namespace bplb {

constexpr int kPrefixNT = 256;
constexpr int kPrefixWarps = kPrefixNT / 32;
// Parameters with at least this many lookups are shared by the whole CTA
// (kCtaBlocks) or by one warp (kWarpBlocks); the rest take one thread each.
constexpr uint32_t kCtaBlocks = 1024;
constexpr uint32_t kWarpBlocks = 32;
constexpr int kMaxHeavy = kPrefixNT;
// Parameters with fewer terms than this are evaluated without the pruning test.
constexpr uint32_t kPruneMinTerms = 4;
// Consecutive parameters per thread in the last phase of CCM1 and BJ1.
constexpr uint32_t kRun = 8;
// FS1's parameters l in [1, 100] (param_range)
constexpr int kFs1Params = 100;

struct PrefixShared {
  int err;
  int skip;  // verdict mode: the instance was decided before this tile
  unsigned long long warp_key[kPrefixWarps];
  long long sums[8];  // n_small, n_big, n_half, n_full, sumw_big, sumw, total big u, unused
  uint32_t wtot[2][kPrefixWarps];
  uint32_t heavy_acc[kMaxHeavy];
  uint32_t heavy_cm[kMaxHeavy];
  uint32_t fs1_cnt[kFs1Params];  // FS1: per parameter, sum_j N(ceil(j c / l'))
  uint32_t fs1_dv[kFs1Params];   //      and the multiples' sum
  uint32_t fs1_cq[kFs1Params], fs1_cr[kFs1Params], fs1_mg[kFs1Params];  // c = cq l' + cr; 2^20 / l' up
  // the tile, decoded by thread 0: DFF (or the u group), table home, FS1 on
  // this tile, the u group's members (bit d), lambda range
  int dec_d, dec_home, dec_fs1, dec_umask;
  long long dec_lam0, dec_lam_end;
  // thread 0's routing of the last decoded instance, reused while the next
  // tiles' instances have the same capacity and route class (route_class;
  // every node of a search-node batch does): the u group merged, FS1 with
  // BJ1, the u group's members and table home, and per DFF its prefix tiles
  // and table home
  long long rc_c;
  int rc_k;
  int rc_merged, rc_wmerged, rc_umask, rc_uhome;
  int rc_nt[kNumDff], rc_home[kNumDff];
  int vb2_mode;  // vb2_table_plan of this u-group tile, with its cut and last l
  long long vb2_kk, vb2_lmax;
  uint32_t minw;  // smallest unpacked size > 0 of the node (transform_bins)
};

// Sum of v over the threads after this one (higher threadIdx.x).  wtot must
// not be in use by another call until the caller's next barrier.
__device__ __forceinline__ uint32_t block_sum_after(uint32_t v, uint32_t *wtot) {
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  uint32_t x = v;  // inclusive suffix within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_down_sync(0xFFFFFFFFu, x, o);
    if (lane + o < 32) x += y;
  }
  if (lane == 0) wtot[warp] = x;
  __syncthreads();
  uint32_t later = 0;
  for (int w = warp + 1; w < kPrefixWarps; ++w) later += wtot[w];
  return x - v + later;
}

// In-place suffix scan of a[0 .. n): a[x] <- sum_{y >= x} a[y], applied once
// or (TWICE) two times.  Thread t scans the contiguous segment
// [t per, t per + per) with per odd (consecutive lanes then hit distinct
// banks); the values entering each segment from above come from block sums
// of the segment totals (TWICE: also of the once-scanned segments' sums).
// n_in, nn_in: what enters a[n - 1] from entries past n (a table scanned in
// parts, the cluster kernel): their sum, and (TWICE) their once-scanned sum.
template <bool TWICE>
__device__ void suffix_scan(int32_t *a, int n, PrefixShared &S, uint32_t n_in = 0u,
                            uint32_t nn_in = 0u) {
  const int per = ((n + kPrefixNT - 1) / kPrefixNT) | 1;
  const int s0 = min(n, (int)threadIdx.x * per), s1 = min(n, s0 + per);
  uint32_t h = 0, m = 0;
  for (int i = s0; i < s1; ++i) {
    const uint32_t v = (uint32_t)a[i];
    h += v;
    if (TWICE) m += v * (uint32_t)(i - s0 + 1);  // this segment's part of the twice-scanned a[s0]
  }
  const uint32_t n_after = block_sum_after(h, S.wtot[0]) + n_in;
  uint32_t nn_after = 0;
  if (TWICE) nn_after = block_sum_after(m + (uint32_t)(s1 - s0) * n_after, S.wtot[1]) + nn_in;
  uint32_t nr = n_after, nnr = nn_after;
  for (int i = s1 - 1; i >= s0; --i) {
    nr += (uint32_t)a[i];
    if (TWICE) {
      nnr += nr;
      a[i] = (int32_t)nnr;
    } else {
      a[i] = (int32_t)nr;
    }
  }
  __syncthreads();
}

// In-place suffix scan of packed count words (low 16 bits: small items at
// u, high 16 bits: big items at u), each word then rewritten as
// (N'(x) mod 2^16) | (Ns(x) << 16) with N' = Ns - Nb.  Every lane's total is
// at most the stream length (< 2^15 on this path), so the packed sums never
// carry from one lane into the other.  n_in: the packed sum of the entries
// past n (a table scanned in parts).
__device__ __forceinline__ void packed_count_scan(uint32_t *a, int n, PrefixShared &S,
                                                  uint32_t n_in = 0u) {
  const int per = ((n + kPrefixNT - 1) / kPrefixNT) | 1;
  const int s0 = min(n, (int)threadIdx.x * per), s1 = min(n, s0 + per);
  uint32_t h = 0;
  for (int i = s0; i < s1; ++i) h += a[i];
  uint32_t run = block_sum_after(h, S.wtot[0]) + n_in;
  for (int i = s1 - 1; i >= s0; --i) {
    run += a[i];
    const uint32_t ns = run & 0xFFFFu, nb = run >> 16;
    a[i] = ((ns - nb) & 0xFFFFu) | (ns << 16);
  }
  __syncthreads();
}

// ---- distributed shared memory of a thread-block cluster ---------------------
// Addresses are 32-bit shared-window addresses: smem_addr of a variable of
// this CTA, cluster_map of that to the same variable in CTA `rank` of the
// cluster (mapa); ld/st/red .shared::cluster then reach any CTA's shared
// memory.  cluster_barrier: every thread of every CTA of the cluster arrives
// (release) and waits (acquire), so that writes before it, local or remote,
// are seen by all reads after it.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ int32_t dsm_ld(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int32_t dsm_ld_s16(uint32_t a) {
  int32_t v;
  asm volatile("ld.shared::cluster.s16 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int4 dsm_ld4(uint32_t a) {
  int4 v;
  asm volatile("ld.shared::cluster.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ unsigned long long dsm_ld64(uint32_t a) {
  unsigned long long v;
  asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void dsm_st(uint32_t a, int32_t v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_st64(uint32_t a, unsigned long long v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void dsm_red_add(uint32_t a, uint32_t v) {
  asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void dsm_red_add64(uint32_t a, unsigned long long v) {
  asm volatile("red.shared::cluster.add.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void dsm_red_or(uint32_t a, uint32_t v) {
  asm volatile("red.shared::cluster.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release;\n\t"
      "barrier.cluster.wait.acquire;" ::: "memory");
}

// ---- table access and thread teams --------------------------------------------
// The evaluators below read a table through an accessor: LocalTab, a plain
// pointer (one CTA's shared memory, or its slice of the global scratch), or
// ClusterTab, a table spread over the shared memory of the CTAs of a
// thread-block cluster (the cluster kernel, bp_lb_cluster.cuh).
// Each gives ld (int32 entry), lo16 (the low 16 bits of an entry,
// sign-extended), ldu (unsigned entry), ld4 (four entries from an entry x
// with phase(x) == 0: one 16-byte load), st, and at(o) (the table starting at
// entry o).  kDeep: the table's loads have a long latency (another CTA's
// shared memory), so that the lookup loops keep more of them in flight.
struct LocalTab {
  static constexpr bool kDeep = false;
  int32_t *p;
  __device__ __forceinline__ int32_t ld(uint32_t x) const { return p[x]; }
  __device__ __forceinline__ int32_t lo16(uint32_t x) const {
    return (int32_t)reinterpret_cast<const int16_t *>(p)[2u * x];
  }
  __device__ __forceinline__ uint32_t ldu(uint32_t x) const {
    return reinterpret_cast<const uint32_t *>(p)[x];
  }
  __device__ __forceinline__ int4 ld4(uint32_t x) const {
    return *reinterpret_cast<const int4 *>(p + x);
  }
  __device__ __forceinline__ void st(uint32_t x, int32_t v) const { p[x] = v; }
  // word offset of entry x within its 16-byte line
  __device__ __forceinline__ uint32_t phase(uint32_t x) const {
    return (uint32_t)(((reinterpret_cast<uintptr_t>(p) >> 2) + x) & 3u);
  }
  __device__ __forceinline__ LocalTab at(uint32_t o) const { return LocalTab{p + o}; }
};

// Entry x of a cluster table lives in CTA x >> kSliceShift of the cluster, at
// word x & (kSliceInts - 1) of its slice; every CTA's slice starts at the same
// shared-memory offset sbase (16-byte aligned), so mapa finds it.  off: the
// cluster-table entry of this table's entry 0.  Every entry the evaluators
// touch lies below the table's length (at most kClusterTableInts); the CTA
// index is clamped all the same, so that no access can leave the cluster.
struct ClusterTab {
  static constexpr bool kDeep = true;
  uint32_t sbase, off;
  const int32_t *lslice;     // this CTA's slice, for reads of its own entries
  uint32_t *acc;             // this CTA's per-parameter accumulators (cluster_harmonic)
  unsigned long long *team;  // kClusterCtas keys: team_max_key's gathering point (CTA 0)
  __device__ __forceinline__ uint32_t addr(uint32_t x) const {
    const uint32_t e = off + x;
    return cluster_map(sbase + ((e & (uint32_t)(kSliceInts - 1)) << 2),
                       min(e >> kSliceShift, (uint32_t)(kClusterCtas - 1)));
  }
  __device__ __forceinline__ int32_t ld(uint32_t x) const { return dsm_ld(addr(x)); }
  __device__ __forceinline__ int32_t lo16(uint32_t x) const { return dsm_ld_s16(addr(x)); }
  __device__ __forceinline__ uint32_t ldu(uint32_t x) const { return (uint32_t)dsm_ld(addr(x)); }
  __device__ __forceinline__ int4 ld4(uint32_t x) const { return dsm_ld4(addr(x)); }
  __device__ __forceinline__ void st(uint32_t x, int32_t v) const { dsm_st(addr(x), v); }
  __device__ __forceinline__ void add(uint32_t x, int32_t v) const {
    dsm_red_add(addr(x), (uint32_t)v);
  }
  __device__ __forceinline__ uint32_t phase(uint32_t x) const { return (off + x) & 3u; }
  __device__ __forceinline__ ClusterTab at(uint32_t o) const {
    return ClusterTab{sbase, off + o, lslice, acc, team};
  }
};

// The threads that share one table's parameters: PARTS CTAs of kPrefixNT
// threads (one CTA, or the CTAs of a cluster), this CTA being number part.
// Loops deal parameters over tid() < kThreads (warps over warp() < kWarps)
// exactly as one CTA's loops deal them over threadIdx.x; sync() is the
// team's barrier.
template <int PARTS>
struct Team {
  static constexpr uint32_t kParts = PARTS;
  static constexpr uint32_t kThreads = PARTS * kPrefixNT;
  static constexpr uint32_t kWarps = PARTS * kPrefixWarps;
  uint32_t part;
  __device__ __forceinline__ uint32_t tid() const { return part * kPrefixNT + threadIdx.x; }
  __device__ __forceinline__ uint32_t warp() const {
    return part * kPrefixWarps + (threadIdx.x >> 5);
  }
  __device__ __forceinline__ void sync() const {
    if constexpr (PARTS == 1) __syncthreads();
    else cluster_barrier();
  }
};
using CtaTeam = Team<1>;

// N' at x: an int32 table (CCM1's own tile) or the low 16 bits of a packed
// count word (the u-group tile, packed_count_scan).
template <bool PACKED, class Tab>
__device__ __forceinline__ int32_t np_at(const Tab &T, uint32_t x) {
  return PACKED ? T.lo16(x) : T.ld(x);
}

// Strided lookup blocks b0, b0 + bs, ... of one parameter (D = CCM1 or BJ1):
// block b is the multiple x = (b + 1) l <= X, its term N'(x) (CCM1, X = U) or
// D(x) at entry 1 + x (BJ1, X = c).  Unrolled by two with explicit bounds (no
// trip-count division).
template <int D, bool PACKED, class Tab>
__device__ __forceinline__ uint32_t block_terms(const Tab &T, uint32_t X, uint32_t l,
                                                uint32_t b0, uint32_t bs) {
  constexpr uint32_t OFF = (D == kBJ1) ? 1u : 0u;
  const uint32_t step = bs * l;
  uint32_t acc = 0;
  uint32_t x = (b0 + 1u) * l;
  if constexpr (Tab::kDeep) {  // eight terms in flight (x + 7 step <= X < 2^21, no wrap)
    for (; x + 7u * step <= X; x += 8u * step) {
      uint32_t s8 = 0;
#pragma unroll
      for (uint32_t e = 0; e < 8u; ++e) s8 += (uint32_t)np_at<PACKED>(T, x + e * step + OFF);
      acc += s8;
    }
  }
  for (; x + step <= X; x += 2u * step)
    acc += (uint32_t)np_at<PACKED>(T, x + OFF) + (uint32_t)np_at<PACKED>(T, x + step + OFF);
  if (x <= X) acc += (uint32_t)np_at<PACKED>(T, x + OFF);
  return acc;
}

// Sum of the terms at the first m multiples of l: N'(i l) (CCM1) or D(i l)
// at entry 1 + i l (BJ1), i = 1 .. m; unrolled by four.
template <int D, bool PACKED, class Tab>
__device__ __forceinline__ uint32_t harmonic_sum(const Tab &T, uint32_t l, uint32_t m) {
  constexpr uint32_t OFF = (D == kBJ1) ? 1u : 0u;
  const uint32_t l2 = 2u * l;
  if (m <= 3u) {
    uint32_t acc = m >= 1u ? (uint32_t)np_at<PACKED>(T, l + OFF) : 0u;
    if (m >= 2u) acc += (uint32_t)np_at<PACKED>(T, l2 + OFF);
    if (m == 3u) acc += (uint32_t)np_at<PACKED>(T, l2 + l + OFF);
    return acc;
  }
  uint32_t acc = 0, x = l + OFF, i = 0;
  if constexpr (Tab::kDeep) {  // eight terms in flight
    for (; i + 8u <= m; i += 8u, x += 4u * l2) {
      uint32_t s8 = 0;
#pragma unroll
      for (uint32_t e = 0; e < 8u; ++e) s8 += (uint32_t)np_at<PACKED>(T, x + e * l);
      acc += s8;
    }
  }
  for (; i + 4u <= m; i += 4u, x += 2u * l2)
    acc += (uint32_t)np_at<PACKED>(T, x) + (uint32_t)np_at<PACKED>(T, x + l) +
           (uint32_t)np_at<PACKED>(T, x + l2) + (uint32_t)np_at<PACKED>(T, x + l2 + l);
  for (; i < m; ++i, x += l) acc += (uint32_t)np_at<PACKED>(T, x);
  return acc;
}

// NN -> D in place (file comment): D(x) = NN(c + 1 - x) - NN(1 + x) at entry
// 1 + x, x in [0, c]; the pair (x, c - x) owns entries 1 + x and c + 1 - x.
// The caller synchronises the team before the entries are read.
template <class Team, class Tab>
__device__ __forceinline__ void nn_to_d(const Tab &T, uint32_t c32, Team tm) {
  for (uint32_t x = tm.tid(); 2u * x <= c32; x += Team::kThreads) {
    const int32_t a = T.ld(1u + x), b = T.ld(c32 + 1u - x);
    T.st(1u + x, b - a);
    T.st(c32 + 1u - x, a - b);
  }
}

// The candidate test (file comment): divide only when S > B f, or for the
// thread's first parameter when there is no floor (B = 0: MT left out of the
// bound, or L1 = 0), so that a bound is kept even when no parameter beats B.
// With the floor L1 a thread may keep nothing: every bound it saw is <= L1,
// which MT's l = 0 holds with the smallest index.  Every sum and denominator
// here is below 2^32 (prefix_handles), so all is 32-bit except the product.
__device__ __forceinline__ void try_key(uint32_t S, uint32_t f, uint32_t g, uint32_t &B,
                                        unsigned long long &best) {
  if ((uint64_t)B * f < (uint64_t)S || (best == 0ull && B == 0u)) {
    const uint32_t q = S / f;
    const uint32_t lb = q + (S != q * f);
    B = max(B, lb);
    best = make_key((int64_t)lb, g);
  }
}

// Pseudo-DFF of the merged u-group tile: MT, RAD2 and CCM1 of one instance
// from one histogram pass (E and packed small/big counts, prefix_u_merged).
constexpr int kPrefixU = kNumDff;

// Per-tile constants of the parameter loops.
struct PrefixEval {
  uint32_t c32, U;
  uint32_t sumw, n_big, n_half, n_full, sumw_big, TB;
  uint32_t B;                // the thread's best bound so far (L1 or 0 at first)
  unsigned long long best;   // the thread's best key
  uint32_t L1;               // pruning cut (prune_ccm1, prune_bj1): L1
  bool prune;                // pruning on and MT part of the bound
};

// Pruning (exact) against L1 = MT's bound at l = 0, which has the smallest
// flattened index, so that a parameter whose bound is at most L1 cannot
// change the maximum or its first argmax.  Upper bounds from the instance's
// sums alone:
//   BJ1: f(w) = p (l - cm) + max(0, rho - cm) <= w (l - cm) / l (w = p l + rho,
//        rho < l), so lb <= ceil(sum w / (q l)) = ceil(sum w / (c - cm));
//   CCM1: floor(u / l) <= u / l for the small items and >= (u - l + 1) / l for
//        the big ones, so with sws = sum_small u, sub = sum_big u,
//        l S <= 2 sws - 2 sub + 2 n_big (l - 1) + q l kS.
__device__ __forceinline__ bool prune_bj1(const PrefixEval &x, uint32_t cm) {
  return x.prune && (uint64_t)x.L1 * (uint64_t)(x.c32 - cm) >= (uint64_t)x.sumw;
}

__device__ __forceinline__ bool prune_ccm1(const PrefixEval &x, uint32_t l, uint32_t q,
                                           uint32_t kS) {
  if (!x.prune) return false;
  const int64_t sws = (int64_t)x.sumw - x.sumw_big - (int64_t)x.n_half * (x.c32 / 2u) -
                      (int64_t)x.n_full * x.c32;
  const int64_t lS = 2 * sws - 2 * (int64_t)x.TB + 2 * (int64_t)x.n_big * (l - 1) +
                     (int64_t)q * l * kS;
  return lS <= 2 * (int64_t)q * l * x.L1;
}

// First l >= l0 with (phase + l) % 4 == 0: entry e of a table starts a
// 16-byte load iff (phase(0) + e) % 4 == 0.
__device__ __forceinline__ uint32_t aligned_from(uint32_t l0, uint32_t phase) {
  return l0 + ((4u - ((phase + l0) & 3u)) & 3u);
}

// MT: S(l) = E(l) + TB + sumw_big + n_half (c/2) + n_full c, f = c; one lookup.
template <class Team, class Tab>
__device__ __forceinline__ void eval_mt(const Tab &E, int64_t lam0, int64_t lam_end,
                                        int64_t c, PrefixEval &x, Team tm) {
  int64_t lo_d, hi_d;
  param_range(kMT, c, lo_d, hi_d);
  const uint32_t gofs = flat_index(kMT, lo_d, c) - (uint32_t)lo_d;
  const uint32_t kS = x.TB + x.sumw_big + x.n_half * (x.c32 / 2u) + x.n_full * x.c32;
  const uint32_t l0 = (uint32_t)lam0, le = (uint32_t)lam_end;
  if (l0 == 0u && tm.tid() == 0 && !x.best) x.best = make_key((int64_t)x.B, gofs);  // l = 0: L1
  for (uint32_t l = l0 + tm.tid(); l < le; l += Team::kThreads)
    try_key((uint32_t)E.ld(min(l, x.U + 1u)) + kS, x.c32, gofs + l, x.B, x.best);
}

// RAD2: n1 = N'(l), n2s = Ns(y), n2b = Ns(y) - N'(y), y = c - 2l + 1; f = c.
template <bool PACKED, class Team, class Tab>
__device__ __forceinline__ void eval_rad2(const Tab &T0, const Tab &T1, int64_t lam0,
                                          int64_t lam_end, int64_t c, PrefixEval &x, Team tm) {
  int64_t lo_d, hi_d;
  param_range(kRAD2, c, lo_d, hi_d);
  const uint32_t gofs = flat_index(kRAD2, lo_d, c) - (uint32_t)lo_d;
  const uint32_t A3 = x.c32 / 3u, B2 = x.c32 / 2u;
  const uint32_t kS = x.n_big * x.c32 + x.n_half * B2 + x.n_full * x.c32;
  for (uint32_t l = (uint32_t)lam0 + tm.tid(); l < (uint32_t)lam_end; l += Team::kThreads) {
    const uint32_t y = min(x.c32 - 2u * l + 1u, x.U + 1u);
    uint32_t n1, n2s, npy;
    if (PACKED) {
      n1 = (uint32_t)np_at<true>(T1, l);
      n2s = T1.ldu(y) >> 16;
      npy = (uint32_t)np_at<true>(T1, y);
    } else {
      n1 = (uint32_t)T0.ld(l);
      n2s = (uint32_t)T1.ld(y);
      npy = (uint32_t)T0.ld(y);
    }
    const uint32_t n2b = n2s - npy;
    try_key(A3 * n1 + (B2 - A3) * n2s - (x.c32 - A3 - B2) * n2b + kS, x.c32, gofs + l, x.B, x.best);
  }
}

// FS1 from the w-domain table (file comment).  Its terms (l', j), j in
// [1, l'] -- 5150 of them for l in [1, 100] -- are cut into equal runs, one per
// thread of the team.  A run walks j (and on to the next l' where one ends)
// with an incremental quotient j c = q l' + r, so that ceil(j c / l') = q +
// [r > 0] and the multiples of the divisibility sum are exactly the terms with
// r = 0 (w = j c / l'); it adds its count and multiples' sums per parameter
// into shared memory (fs1_accumulate), after which thread l - lo of one CTA
// forms S(l) in 64 bits and keeps the key (fs1_finish; the first parameters
// its thread meets).  With c < 2^20 on this path every j c fits 32 bits; the
// count sum, at most 101 (sum w) / c, is below 2^32 by prefix_home, and the
// multiples' sum is at most sum w.
__device__ __forceinline__ uint32_t tri(uint32_t m) { return m * (m + 1u) / 2u; }

template <class Team, class Tab>
__device__ __forceinline__ void fs1_accumulate(const Tab &T, int64_t c, PrefixShared &S, Team tm) {
  int64_t lo_d, hi_d;
  param_range(kFS1, c, lo_d, hi_d);
  const uint32_t lo = (uint32_t)lo_d, hi = (uint32_t)hi_d;
  const uint32_t c32 = (uint32_t)c;
  const uint32_t base = tri(lo);  // term index of (l' = lo + 1, j = 1), plus base
  const uint32_t total = tri(hi + 1u) - base;
  const uint32_t per = (total + Team::kThreads - 1) / Team::kThreads;
  uint32_t p = tm.tid() * per;
  const uint32_t pe = min(total, p + per);
  if (p < pe) {
    // the run's first term: l = the largest m with tri(m) <= p + base
    const uint32_t P = p + base;
    uint32_t l = (uint32_t)((sqrtf(8.0f * (float)P + 1.0f) - 1.0f) * 0.5f);
    while (tri(l + 1u) <= P) ++l;
    while (tri(l) > P) --l;
    uint32_t j = P - tri(l) + 1u;
    while (p < pe) {
      const uint32_t lp = l + 1u;
      // j c = q l' + r from the per-parameter constants: j cr < l'^2 <= 10201,
      // so its quotient by l' from the rounded-up 2^20 / l' is within one
      const uint32_t cq = S.fs1_cq[l - lo], cr = S.fs1_cr[l - lo];
      const uint32_t n = j * cr;
      uint32_t t = (n * S.fs1_mg[l - lo]) >> 20;
      uint32_t r = n - t * lp;
      if ((int32_t)r < 0) {
        --t;
        r += lp;
      }
      uint32_t q = j * cq + t;
      const uint32_t j0 = j, jend = min(lp, j + (pe - p) - 1u);
      uint32_t cnt = 0, dv = 0;
      for (;;) {
        const uint32_t xj = q + (r != 0u);  // in [1, c]
        const int32_t nx = T.ld(xj) - T.ld(xj + 1u);
        cnt += (uint32_t)nx;
        if (r == 0u) {  // c divides xj l': xj's items map to xj l
          const int32_t nx1 = (xj < c32) ? T.ld(xj + 1u) - T.ld(xj + 2u) : 0;  // N(c + 1) = 0
          dv += xj * (uint32_t)(nx - nx1);
        }
        if (j == jend) break;
        ++j;
        q += cq;
        r += cr;
        if (r >= lp) {
          r -= lp;
          ++q;
        }
      }
      atomicAdd(&S.fs1_cnt[l - lo], cnt);
      if (dv != 0u) atomicAdd(&S.fs1_dv[l - lo], dv);
      p += jend - j0 + 1u;
      ++l;
      j = 1u;
    }
  }
}

// FS1's keys from the sums fs1_accumulate left in S (after the team's
// barrier): thread l - lo takes parameter l.
__device__ __forceinline__ void fs1_finish(int64_t c, PrefixEval &x, const PrefixShared &S) {
  int64_t lo_d, hi_d;
  param_range(kFS1, c, lo_d, hi_d);
  const uint32_t lo = (uint32_t)lo_d, hi = (uint32_t)hi_d;
  const uint32_t gofs = flat_index(kFS1, lo_d, c) - lo;
  const uint32_t c32 = x.c32;
  if (threadIdx.x <= hi - lo) {
    const uint32_t l = lo + threadIdx.x;
    const uint64_t Sv = (uint64_t)c32 * S.fs1_cnt[threadIdx.x] - S.fs1_dv[threadIdx.x];
    const uint64_t f = (uint64_t)c32 * l;
    if ((uint64_t)x.B * f < Sv || (x.best == 0ull && x.B == 0u)) {
      const uint64_t qv = Sv / f;
      const uint32_t lb = (uint32_t)(qv + (Sv != qv * f));
      x.B = max(x.B, lb);
      x.best = make_key((int64_t)lb, gofs + l);
    }
  }
}

// CCM1 / BJ1: the lookups of parameter l fall like X / l, so heavy parameters
// are shared by the CTA, medium ones by a warp, the rest take a thread each.
// (A cluster's tables take cluster_harmonic instead.)
template <int D, bool PACKED, class Team, class Tab>
__device__ void eval_harmonic(const Tab &T0, int64_t lam0, int64_t lam_end, int64_t c,
                              PrefixEval &x, PrefixShared &S, Team tm) {
  const int tid = threadIdx.x;
  const uint32_t c32 = x.c32, U = x.U;
  int64_t lo_d, hi_d;
  param_range(D, c, lo_d, hi_d);
  const uint32_t gofs = flat_index(D, lo_d, c) - (uint32_t)lo_d;
  //   CCM1: S = 2 acc + q kS, f = 2q;   BJ1: S = acc (sum w when cm = 0), f = q (l - cm)
  const uint32_t kS = (D == kCCM1) ? 2u * x.n_big + x.n_half + 2u * x.n_full : x.sumw;
  const uint32_t le = (uint32_t)lam_end;
  const uint32_t X = (D == kCCM1) ? U : c32;
  const int64_t cta_end = max(lam0, min(lam_end, min((int64_t)(X / kCtaBlocks) + 1, lam0 + kMaxHeavy)));
  const int64_t warp_end = max(cta_end, min(lam_end, (int64_t)(X / kWarpBlocks) + 1));
  const int lane = (int)lane_id();
  const uint32_t gwarp = tm.warp(), gtid = tm.tid();
  constexpr uint32_t W = Team::kWarps;
  auto finish = [&](uint32_t l, uint32_t q, uint32_t acc) {
    uint32_t Sv, f;
    if (D == kCCM1) {
      Sv = 2u * acc + q * kS;
      f = 2u * q;
    } else {
      const uint32_t cm = c32 - q * l;
      Sv = cm == 0u ? kS : acc;
      f = q * (l - cm);  // <= c
    }
    try_key(Sv, f, gofs + l, x.B, x.best);
  };

  // ---- parameters shared by the whole CTA ---------------------------------------
  // pruned parameters (prune_bj1, prune_ccm1) are skipped altogether
  auto pruned = [&](uint32_t l, uint32_t q, uint32_t cm) {
    return D == kBJ1 ? prune_bj1(x, cm) : prune_ccm1(x, l, q, kS);
  };
  constexpr uint32_t kPruned = 0xFFFFFFFFu;  // heavy_cm marker (cm < l otherwise)
  const int ncta = (int)(cta_end - lam0);
  if (ncta > 0) {
    if (tid < ncta) {
      const uint32_t l = (uint32_t)(lam0 + tid);
      const uint32_t q = c32 / l, cm = c32 - q * l;
      S.heavy_cm[tid] = pruned(l, q, cm) ? kPruned : cm;
      S.heavy_acc[tid] = 0u;
    }
    __syncthreads();
    for (int i = 0; i < ncta; ++i) {
      const uint32_t l = (uint32_t)(lam0 + i);
      const uint32_t cm = S.heavy_cm[i];
      if (cm == kPruned || (D == kBJ1 && cm == 0u)) continue;  // BJ1, cm = 0: S = sum w
      const uint32_t part = __reduce_add_sync(
          0xFFFFFFFFu, block_terms<D, PACKED>(T0, X, l, (uint32_t)tid, kPrefixNT));
      if (lane == 0 && part != 0u) atomicAdd(&S.heavy_acc[i], part);
    }
    __syncthreads();
    if (tid < ncta && S.heavy_cm[tid] != kPruned) {
      const uint32_t l = (uint32_t)(lam0 + tid);
      finish(l, c32 / l, S.heavy_acc[tid]);
    }
  }

  // ---- parameters shared by one warp --------------------------------------------
  // Round i gives warp w (of the team's W) the parameter cta_end + W i + w (i
  // even) or + W - 1 - w (i odd); lane t of a batch of 32 rounds owns the t-th
  // one: it computes its quotient, broadcasts cm, and keeps the warp's sum.
  {
    const int64_t nwarp = warp_end - cta_end;
    const int64_t rounds = (nwarp + W - 1) / W;
    for (int64_t r0 = 0; r0 < rounds; r0 += 32) {
      const int64_t ri = r0 + lane;
      const int64_t my_l = cta_end + ri * W + ((ri & 1) ? W - 1 - gwarp : gwarp);
      const bool in_range = ri < rounds && my_l < warp_end;
      const uint32_t ml = in_range ? (uint32_t)my_l : 1u;
      const uint32_t mq = c32 / ml;
      const uint32_t mcm = c32 - mq * ml;
      const bool mine_ok = in_range && !pruned(ml, mq, mcm);
      uint32_t mine = 0;
      const int cnt = (int)min((int64_t)32, rounds - r0);
      for (int t = 0; t < cnt; ++t) {
        const uint32_t l = __shfl_sync(0xFFFFFFFFu, ml, t);
        const uint32_t cm = __shfl_sync(0xFFFFFFFFu, mcm, t);
        const bool ok = __shfl_sync(0xFFFFFFFFu, (int)mine_ok, t) != 0;
        if (!ok || (D == kBJ1 && cm == 0u)) continue;
        const uint32_t part = __reduce_add_sync(
            0xFFFFFFFFu, block_terms<D, PACKED>(T0, X, l, (uint32_t)lane, 32u));
        if (lane == t) mine = part;
      }
      if (mine_ok) finish(ml, mq, mine);
    }
  }

  // ---- one thread per run of kRun parameters -----------------------------------------
  // Warp blocks of 32 kRun consecutive lambdas from warp_end on; round i gives
  // warp w the block i W + w (i even) or + W - 1 - w (i odd), so that the
  // warps' loads balance, and lane t of it the lambdas
  // base + t + 32 k, k < kRun: a thread's parameters increase, and at each
  // step the warp reads consecutive lambdas' terms.  One division per run for
  // q = floor(c / l) and m = floor(X / l) (the number of terms), decrements
  // after it.  The pruning tests (prune_bj1, prune_ccm1) in their linear forms
  // with per-thread constants, and only for parameters with many terms.
  {
    const int64_t A0 = 2 * ((int64_t)x.sumw - x.sumw_big - (int64_t)x.n_half * (c32 / 2u) -
                            (int64_t)x.n_full * c32 - (int64_t)x.TB - (int64_t)x.n_big);
    const int64_t A1 = 2 * (int64_t)x.n_big;
    const int64_t A2 = 2 * (int64_t)x.L1 - (int64_t)kS;
    constexpr uint32_t kBlock = 32u * kRun;
    // BJ1's l > c / 2 (q = 1) are taken below, four at a time
    const uint32_t lq1 = (D == kBJ1) ? max((uint32_t)warp_end, min(le, c32 / 2u + 1u)) : le;
    bool odd = false;
    for (uint32_t r0 = (uint32_t)warp_end; r0 < lq1; r0 += kBlock * W, odd = !odd) {
      const uint32_t wb = odd ? W - 1u - gwarp : gwarp;
      const uint32_t l0 = r0 + wb * kBlock + (uint32_t)lane;
      if (l0 >= lq1) continue;
      uint32_t q = c32 / l0, m = (D == kCCM1) ? U / l0 : 0u;
      for (uint32_t l = l0; l < lq1 && l < l0 + kBlock; l += 32u) {
        while (q * l > c32) --q;  // q l <= c (l0 + kBlock) / l0 < 2^32 here
        if (D == kCCM1) {
          while (m * l > U) --m;
        } else {
          m = q;
        }
        if (x.prune && m >= kPruneMinTerms) {
          const bool cut = (D == kBJ1) ? (uint64_t)x.L1 * (uint64_t)(q * l) >= (uint64_t)x.sumw
                                       : A0 + A1 * (int64_t)l <= (int64_t)(q * l) * A2;
          if (cut) continue;
        }
        uint32_t acc = 0;
        if (D == kCCM1 || q * l != c32) acc = harmonic_sum<D, PACKED>(T0, l, m);
        finish(l, q, acc);
      }
    }
    // BJ1, q = 1: S = D(l) at entry 1 + l (D(c) = sum w covers c mod l = 0),
    // f = 2l - c.  Parameters from la (entry 1 + la 16-byte aligned) go four
    // to a thread per step, one 16-byte load each; the few before la one each.
    if (D == kBJ1 && lq1 < le) {
      const uint32_t la = min(le, aligned_from(lq1, T0.phase(1)));  // entry 1 + la aligned
      if (lq1 + gtid < la) {
        const uint32_t l = lq1 + gtid;
        try_key((uint32_t)T0.ld(1u + l), 2u * l - c32, gofs + l, x.B, x.best);
      }
      for (uint32_t l = la + 4u * gtid; l < le; l += 4u * Team::kThreads) {
        if (l + 3u < le) {
          const int4 v = T0.ld4(1u + l);
          try_key((uint32_t)v.x, 2u * l - c32, gofs + l, x.B, x.best);
          try_key((uint32_t)v.y, 2u * l + 2u - c32, gofs + l + 1u, x.B, x.best);
          try_key((uint32_t)v.z, 2u * l + 4u - c32, gofs + l + 2u, x.B, x.best);
          try_key((uint32_t)v.w, 2u * l + 6u - c32, gofs + l + 3u, x.B, x.best);
        } else {
          for (uint32_t e = l; e < le; ++e) try_key((uint32_t)T0.ld(1u + e), 2u * e - c32, gofs + e, x.B, x.best);
        }
      }
    }
  }
}

// Quotient n / l for n < 2^21, l >= 1: a float estimate (error below one) and
// one correction.
__device__ __forceinline__ uint32_t small_div(uint32_t n, uint32_t l) {
  uint32_t q = (uint32_t)((float)n * __frcp_rn((float)l));
  if (q * l > n) --q;
  else if ((q + 1u) * l <= n) ++q;
  return q;
}

constexpr uint32_t kOwnChunk = 8192;                       // parameters per chunk
constexpr uint32_t kOwnPerCta = kOwnChunk / kClusterCtas;  // accumulators per CTA
constexpr int64_t kOwnBytes = 4 * (int64_t)kOwnPerCta;

// CCM1 / BJ1 with the cluster's table: S(l) = sum_{i=1}^{m} T(i l + OFF) (m =
// floor(U / l) for CCM1, q = floor(c / l) for BJ1, OFF = 1 for BJ1) is the
// sum over the CTAs of the terms whose entry lies in each CTA's own slice,
// read there from local shared memory; each CTA adds its partial sum into the
// accumulator of the parameter's owner (red.shared::cluster), and after a
// cluster barrier the owner forms the bound.  Parameters go in chunks of
// kOwnChunk, owner of parameter cb + j the CTA j / kOwnPerCta, its thread
// j % kPrefixNT (increasing within a thread, as the key rule wants).
// Parameters of one warp-sized local run or more (l <= kSliceInts / 32) are
// shared by a warp, the rest take a thread each.
template <int D, bool PACKED, class Team>
__device__ void cluster_harmonic(const ClusterTab &T, int64_t lam0, int64_t lam_end, int64_t c,
                                 PrefixEval &x, Team tm) {
  constexpr uint32_t OFF = (D == kBJ1) ? 1u : 0u;
  const int32_t *slice = T.lslice;
  uint32_t *acc_own = T.acc;
  const uint32_t off = T.off;
  const int tid = threadIdx.x;
  const uint32_t rank = tm.part;
  const uint32_t c32 = x.c32, U = x.U;
  const uint32_t X = (D == kCCM1) ? U : c32;
  int64_t lo_d, hi_d;
  param_range(D, c, lo_d, hi_d);
  const uint32_t gofs = flat_index(D, lo_d, c) - (uint32_t)lo_d;
  const uint32_t kS = (D == kCCM1) ? 2u * x.n_big + x.n_half + 2u * x.n_full : x.sumw;
  // this CTA's entries of the table: table indices [ta, tb)
  const uint32_t s0 = rank << kSliceShift;
  const uint32_t s1 = s0 + (uint32_t)kSliceInts;
  const uint32_t ta = s0 > off ? s0 - off : 0u;
  const uint32_t tb = s1 > off ? min(s1 - off, X + OFF + 1u) : 0u;
  auto tv = [&](uint32_t t) -> uint32_t {  // table entry t, local
    const uint32_t e = off + t - s0;
    return PACKED ? (uint32_t)(int32_t)reinterpret_cast<const int16_t *>(slice)[2u * e]
                  : (uint32_t)slice[e];
  };
  auto pruned = [&](uint32_t l, uint32_t q, uint32_t cm) {
    return D == kBJ1 ? prune_bj1(x, cm) : prune_ccm1(x, l, q, kS);
  };
  // terms i in [1, m] with entry i l + OFF in [ta, tb): i in [ilo, ihi]
  auto local_range = [&](uint32_t l, uint32_t m, uint32_t &ilo, uint32_t &ihi) {
    ilo = ta > OFF ? small_div(ta - OFF + l - 1u, l) : 1u;
    if (ilo < 1u) ilo = 1u;
    ihi = tb > OFF + 1u ? min(m, small_div(tb - 1u - OFF, l)) : 0u;
  };
  const uint32_t lheavy = (uint32_t)(kSliceInts / 32);
  const int lane = (int)lane_id(), warp = tid >> 5;
  for (int64_t cb = lam0; cb < lam_end; cb += kOwnChunk) {
    const uint32_t ce = (uint32_t)min(lam_end, cb + (int64_t)kOwnChunk);
    const uint32_t c0 = (uint32_t)cb;
    // ---- partial sums of this CTA's terms into the owners' accumulators ----
    const uint32_t hend = min(ce, max(c0, lheavy + 1u));  // warp-shared parameters [c0, hend)
    for (uint32_t l = c0 + (uint32_t)warp; l < hend; l += kPrefixWarps) {
      const uint32_t q = c32 / l, cm = c32 - q * l;
      if (pruned(l, q, cm) || (D == kBJ1 && cm == 0u)) continue;
      const uint32_t m = (D == kCCM1) ? U / l : q;
      uint32_t ilo, ihi;
      local_range(l, m, ilo, ihi);
      uint32_t s = 0;
      for (uint32_t i = ilo + (uint32_t)lane; i <= ihi; i += 32u) s += tv(i * l + OFF);
      s = __reduce_add_sync(0xFFFFFFFFu, s);
      if (lane == 0 && s != 0u) {
        const uint32_t j = l - c0;
        dsm_red_add(cluster_map(smem_addr(&acc_own[j % kOwnPerCta]), j / kOwnPerCta), s);
      }
    }
    // parameters up to a slice's length: each thread its own, every CTA
    // its slice's terms of it
    const uint32_t lsl = min(ce, max(hend, (uint32_t)kSliceInts + 1u));
    for (uint32_t l = hend + (uint32_t)tid; l < lsl; l += kPrefixNT) {
      const uint32_t q = small_div(c32, l), cm = c32 - q * l;
      if (pruned(l, q, cm) || (D == kBJ1 && cm == 0u)) continue;
      const uint32_t m = (D == kCCM1) ? small_div(U, l) : q;
      // no term in this CTA's entries: the first lies past them or the last before
      if (m == 0u || l + OFF >= tb || m * l + OFF < ta) continue;
      uint32_t ilo, ihi;
      local_range(l, m, ilo, ihi);
      uint32_t s = 0;
      for (uint32_t i = ilo; i <= ihi; ++i) s += tv(i * l + OFF);
      if (s != 0u) {
        const uint32_t j = l - c0;
        dsm_red_add(cluster_map(smem_addr(&acc_own[j % kOwnPerCta]), j / kOwnPerCta), s);
      }
    }
    // parameters longer than a slice: at most one multiple i l of each in
    // this CTA's entries, so the CTA walks i and, for each, the parameters
    // with i l + OFF in its entries -- only those -- one term each (whether
    // pruned or not: the owner decides)
    if (lsl < ce && tb > ta && tb > OFF + 1u) {
      const uint32_t imax = (tb - 1u - OFF) / lsl;
      for (uint32_t i = 1u; i <= imax; ++i) {
        const uint32_t l0 = max(lsl, ta > OFF ? (ta - OFF + i - 1u) / i : 0u);
        const uint32_t l1 = min(min(ce - 1u, (tb - 1u - OFF) / i), X / i);
        for (uint32_t l = l0 + (uint32_t)tid; l <= l1; l += kPrefixNT) {
          const uint32_t s = tv(i * l + OFF);
          if (s != 0u) {
            const uint32_t j = l - c0;
            dsm_red_add(cluster_map(smem_addr(&acc_own[j % kOwnPerCta]), j / kOwnPerCta), s);
          }
        }
      }
    }
    cluster_barrier();  // every partial in its owner
    // ---- the owner forms the bounds of its parameters ----------------------------
    for (uint32_t j = rank * kOwnPerCta + (uint32_t)tid; j < (rank + 1u) * kOwnPerCta; j += kPrefixNT) {
      const uint32_t l = c0 + j;
      const uint32_t acc = acc_own[j - rank * kOwnPerCta];
      acc_own[j - rank * kOwnPerCta] = 0u;
      if (l >= ce) continue;
      const uint32_t q = small_div(c32, l), cm = c32 - q * l;
      if (pruned(l, q, cm)) continue;
      uint32_t Sv, f;
      if (D == kCCM1) {
        Sv = 2u * acc + q * kS;
        f = 2u * q;
      } else {
        Sv = cm == 0u ? kS : acc;
        f = q * (l - cm);
      }
      try_key(Sv, f, gofs + l, x.B, x.best);
    }
    cluster_barrier();  // accumulators cleared before the next chunk's sums
  }
}

// VB2 on the u group's tile.  For u >= 1, ceil(l u / c) counts the j in
// [0, l) with u >= floor(j c / l) + 1, so summed with sign over the small and
// big items VB2's accumulator is sum_j N'(floor(j c / l) + 1), the terms
// vanishing past U: about l / 2 lookups of the packed table per parameter.
// That is only cheap for small l, so the tile takes VB2 when pruning leaves
// only such parameters: every parameter that may matter satisfies
// G(l) = alpha l + beta > 0 (vb2_range_may_exceed), and with alpha < 0 those
// are l <= lmax.  Returns 0 (VB2 stays with its kernel), 1 (evaluate l in
// [2, lmax] here) or 2 (no VB2 parameter can matter); the cut kk is k in
// verdict mode, else L1 (MT in the bound), clamped to the stream length.
// `budget`: the most lookups the tile takes on (kVb2TableTerms per CTA of
// its team).
constexpr int64_t kVb2TableTerms = 1 << 16;  // lookups per CTA at most
// A cluster unit's second plan (late_vb2_plan; cluster_vb2, local lookups,
// most of them in the three or four CTAs that hold the count table): above
// about 2^21 lookups the unit takes longer than the generic kernel's VB2
// tiles, which spread over every SM.
constexpr int64_t kClusterVb2Terms = 1 << 21;

// L1 may be any cut known from keys already found (late_vb2_plan).
template <int MODE>
__device__ __forceinline__ int vb2_table_plan(const EvalArgs &A, const InstView &I,
                                              const PrefixShared &S, uint32_t L1,
                                              int64_t vb2_cap_hi, int64_t budget, int64_t &kk,
                                              int64_t &lmax) {
  const int64_t c = I.c;
  if (!(A.prune || A.verdict) || ((A.dff_off >> kVB2) & 1u) || !A.vb2_on || c < 2) return 0;
  const int64_t cut = A.verdict ? I.k : ((A.dff_off & 1u) ? -1 : (int64_t)L1);
  if (cut < 0) return 0;
  kk = min(cut, stream_len<MODE>(I));
  const int64_t ns = S.sums[0], nb = S.sums[1], nh = S.sums[2], nf = S.sums[3];
  const int64_t swb = S.sums[4], sw = S.sums[5];
  const int64_t Dd = (sw - swb - nh * (c / 2) - nf * c) - (nb * c - swb);
  const int64_t K = 2 * nb + nh + 2 * nf;
  const int64_t alpha = 2 * Dd - c * (2 * kk - K);
  const int64_t beta = 2 * ns * (c - 1) + c * (2 * kk - K) - c * (2 * ns - 2 * nb + 1) + 2;
  if (alpha >= 0) return (alpha * c + beta <= 0) ? 2 : 0;
  if (2 * alpha + beta <= 0) return 2;
  lmax = min(c, (beta - 1) / (-alpha));
  if (A.vb2_hi != nullptr) {  // the cap of Sec. 4: no parameter above it
    lmax = min(lmax, vb2_cap_hi);
    if (lmax < 2) return 2;
  }
  const int64_t U = (c - 1) / 2;
  return (U * lmax * lmax / (2 * c) + lmax <= budget) ? 1 : 0;
}

// VB2's parameters l in [2, lmax] from the packed count table T (entry x:
// N'(x) in its low 16 bits), one thread each: round i gives thread t the
// parameter 2 + i kPrefixNT + t (i even) or + kPrefixNT - 1 - t (i odd), so
// that the threads' term counts (about l / 2) balance and each thread's
// parameters increase.  The terms walk j with an incremental quotient
// j c = q l + r (no division but c / l per parameter).  Every l in the range
// is evaluated exactly (the range is a relaxation of the parameters that can
// matter; the others only cost their lookups).
template <class Team, class Tab>
__device__ __forceinline__ void eval_vb2_table(const Tab &T, int64_t c, PrefixEval &x,
                                               const PrefixShared &S, int64_t lmax, Team tm) {
  const uint32_t c32 = x.c32, U = x.U;
  const uint32_t gofs = flat_index(kVB2, 2, c) - 2u;
  const int64_t ns = S.sums[0], nb = S.sums[1];
  const int64_t K = 2 * nb + S.sums[2] + 2 * S.sums[3];
  const uint32_t n = (uint32_t)lmax - 1u;  // parameters 2 .. lmax
  bool odd = false;
  for (uint32_t r0 = 0; r0 < n; r0 += Team::kThreads, odd = !odd) {
    const uint32_t p = r0 + (odd ? Team::kThreads - 1u - tm.tid() : tm.tid());
    if (p >= n) continue;
    const uint32_t l = 2u + p;
    const uint32_t cq = c32 / l, cr = c32 - cq * l;
    uint32_t q = 0, r = 0;
    int32_t acc = 0;
    while (q < U) {  // the term's entry q + 1 <= U
      acc += np_at<true>(T, q + 1u);
      q += cq;
      r += cr;
      if (r >= l) {
        r -= l;
        ++q;
      }
    }
    const int64_t Sv = 2 * ((int64_t)acc - ns + nb) + (int64_t)(l - 1u) * K;  // >= 0
    const uint64_t f = 2u * (l - 1u);
    if ((uint64_t)x.B * f < (uint64_t)Sv || (x.best == 0ull && x.B == 0u)) {
      const uint32_t lb = (uint32_t)(((uint64_t)Sv + f - 1u) / f);
      x.B = max(x.B, lb);
      x.best = make_key((int64_t)lb, gofs + l);
    }
  }
}

// VB2 from a cluster's packed count table by owner-computes, as
// cluster_harmonic does CCM1 and BJ1: parameter l's terms are the entries
// floor(j c / l) + 1 <= U, j = 0, 1, ... (eval_vb2_table), increasing with j,
// so those in this CTA's slice are the terms of one run of j, which the CTA
// walks from its first with the incremental quotient.  With t0 the slice's
// first table index, that first j is j0 = ceil((t0 - 1) l / c), and j0 c =
// (t0 - 1) l + d with 0 <= d < c gives floor(j0 c / l) = t0 - 1 +
// floor(d / l).  Parameters of about 80 terms a slice or more (l >=
// kVb2WarpMin) take a warp, whose lane t walks j0 + t, j0 + t + 32, ...; the
// others a thread each.  Each CTA adds its partial sums into the owners'
// accumulators (chunks of kOwnChunk parameters, owner of parameter cb + j the
// CTA j / kOwnPerCta), and the owner forms the bounds as eval_vb2_table
// does.  The accumulators hold wrapping 32-bit sums of the signed counts.
constexpr uint32_t kVb2WarpMin = 512;

// Quotient n / l for n < 2^24 and a quotient below 2^21: the float estimate
// is within one of it, so one correction each way.
__device__ __forceinline__ uint32_t est_div(uint32_t n, uint32_t l) {
  uint32_t q = (uint32_t)((float)n * __frcp_rn((float)l));
  if (q * l > n) --q;
  else if ((q + 1u) * l <= n) ++q;
  return q;
}

template <class Team>
__device__ void cluster_vb2(const ClusterTab &T, int64_t c, PrefixEval &x, const PrefixShared &S,
                            int64_t lmax, Team tm) {
  const int16_t *lo16 = reinterpret_cast<const int16_t *>(T.lslice);
  uint32_t *acc_own = T.acc;
  const uint32_t off = T.off;
  const int tid = threadIdx.x;
  const uint32_t rank = tm.part;
  const uint32_t c32 = x.c32, U = x.U;
  const uint32_t gofs = flat_index(kVB2, 2, c) - 2u;
  const int64_t ns = S.sums[0], nb = S.sums[1];
  const int64_t K = 2 * nb + S.sums[2] + 2 * S.sums[3];
  // this CTA's table indices [ta, tb) within the terms' [1, U]
  const uint32_t s0 = rank << kSliceShift;
  const uint32_t s1 = s0 + (uint32_t)kSliceInts;
  const uint32_t ta = max(s0 > off ? s0 - off : 0u, 1u);
  const uint32_t tb = s1 > off ? min(s1 - off, U + 1u) : 0u;
  const bool local = ta < tb;
  const float inv_c = 1.0f / (float)c32;
  // d of parameter l (file comment); j0 from a float estimate, corrected
  // against the exact 64-bit products (the estimate is within one of it)
  auto first_d = [&](uint32_t l) -> uint32_t {
    const uint64_t P = (uint64_t)(ta - 1u) * l;
    uint64_t j0 = (uint64_t)((float)(ta - 1u) * (float)l * inv_c);
    if (j0 * c32 < P) ++j0;
    if (j0 * c32 < P) ++j0;
    if (j0 > 0u && (j0 - 1u) * c32 >= P) --j0;
    if (j0 > 0u && (j0 - 1u) * c32 >= P) --j0;
    return (uint32_t)(j0 * c32 - P);
  };
  auto tv = [&](uint32_t t) -> uint32_t {  // N'(t), from this CTA's slice
    return (uint32_t)(int32_t)lo16[2u * (off + t - s0)];
  };
  auto add_owner = [&](uint32_t j, uint32_t s) {
    dsm_red_add(cluster_map(smem_addr(&acc_own[j % kOwnPerCta]), j / kOwnPerCta), s);
  };
  const int lane = (int)lane_id(), warp = tid >> 5;
  const uint32_t lend = (uint32_t)lmax + 1u;  // parameters [2, lmax]
  for (uint32_t cb = 2u; cb < lend; cb += kOwnChunk) {
    const uint32_t ce = min(lend, cb + kOwnChunk);
    // ---- partial sums of this CTA's terms into the owners' accumulators ----
    const uint32_t wbeg = min(ce, max(cb, kVb2WarpMin));  // thread parameters [cb, wbeg)
    if (local) {
      const uint32_t n = wbeg - cb;
      bool odd = false;
      for (uint32_t r0 = 0; r0 < n; r0 += kPrefixNT, odd = !odd) {
        const uint32_t p = r0 + (odd ? kPrefixNT - 1u - (uint32_t)tid : (uint32_t)tid);
        if (p >= n) continue;
        const uint32_t l = cb + p;
        const uint32_t d = first_d(l);
        const uint32_t dq = est_div(d, l);
        uint32_t q = ta - 1u + dq, r = d - dq * l;
        const uint32_t cq = est_div(c32, l), cr = c32 - cq * l;
        uint32_t s = 0;
        while (q + 1u < tb) {
          s += tv(q + 1u);
          q += cq;
          r += cr;
          if (r >= l) {
            r -= l;
            ++q;
          }
        }
        if (s != 0u) add_owner(l - cb, s);
      }
      const uint32_t c32x = 32u * c32;
      for (uint32_t l = wbeg + (uint32_t)warp; l < ce; l += kPrefixWarps) {
        const uint32_t dt = first_d(l) + (uint32_t)lane * c32;  // < 32 c < 2^24
        const uint32_t dq = est_div(dt, l);
        uint32_t q = ta - 1u + dq, r = dt - dq * l;
        const uint32_t cq = est_div(c32x, l), cr = c32x - cq * l;
        uint32_t s = 0;
        while (q + 1u < tb) {
          s += tv(q + 1u);
          q += cq;
          r += cr;
          if (r >= l) {
            r -= l;
            ++q;
          }
        }
        s = __reduce_add_sync(0xFFFFFFFFu, s);
        if (lane == 0 && s != 0u) add_owner(l - cb, s);
      }
    }
    cluster_barrier();  // every partial in its owner
    // ---- the owner forms the bounds of its parameters ----------------------------
    for (uint32_t j = rank * kOwnPerCta + (uint32_t)tid; j < (rank + 1u) * kOwnPerCta; j += kPrefixNT) {
      const uint32_t l = cb + j;
      const int32_t acc = (int32_t)acc_own[j - rank * kOwnPerCta];
      acc_own[j - rank * kOwnPerCta] = 0u;
      if (l >= ce) continue;
      const int64_t Sv = 2 * ((int64_t)acc - ns + nb) + (int64_t)(l - 1u) * K;  // >= 0
      const uint64_t f = 2u * (l - 1u);
      if ((uint64_t)x.B * f < (uint64_t)Sv || (x.best == 0ull && x.B == 0u)) {
        const uint32_t lb = (uint32_t)(((uint64_t)Sv + f - 1u) / f);
        x.B = max(x.B, lb);
        x.best = make_key((int64_t)lb, gofs + l);
      }
    }
    cluster_barrier();  // accumulators cleared before the next chunk's sums
  }
}

// A team of several CTAs: every CTA but 0 adds its FS1 sums into CTA 0's
// (after the CTA's barrier; the team's barrier follows).
template <class Team>
__device__ __forceinline__ void fs1_gather(PrefixShared &S, Team tm) {
  if (tm.part != 0u && threadIdx.x < kFs1Params) {
    const uint32_t t = threadIdx.x;
    if (S.fs1_cnt[t] != 0u) dsm_red_add(cluster_map(smem_addr(&S.fs1_cnt[t]), 0), S.fs1_cnt[t]);
    if (S.fs1_dv[t] != 0u) dsm_red_add(cluster_map(smem_addr(&S.fs1_dv[t]), 0), S.fs1_dv[t]);
  }
}

// The largest of the team's threads' keys, returned to every thread (team
// barriers inside; warp_key, and for a cluster team[0 .. kClusterCtas) in
// every CTA, as scratch).
template <class Team>
__device__ __forceinline__ unsigned long long team_max_key(unsigned long long key, PrefixShared &S,
                                                           unsigned long long *team, Team tm) {
  key = warp_max_u64(key);
  if (lane_id() == 0) S.warp_key[threadIdx.x >> 5] = key;
  __syncthreads();
  unsigned long long m = 0ull;
  for (int w = 0; w < kPrefixWarps; ++w) m = S.warp_key[w] > m ? S.warp_key[w] : m;
  if constexpr (Team::kParts > 1) {
    if (threadIdx.x == 0) dsm_st64(cluster_map(smem_addr(&team[tm.part]), 0), m);
    tm.sync();
    if (threadIdx.x < Team::kParts)
      S.warp_key[threadIdx.x] = dsm_ld64(cluster_map(smem_addr(&team[threadIdx.x]), 0));
    __syncthreads();
    m = 0ull;
    for (uint32_t r = 0; r < Team::kParts; ++r) m = S.warp_key[r] > m ? S.warp_key[r] : m;
  }
  __syncthreads();  // warp_key free again
  return m;
}

// The u group's second VB2 plan, after MT, RAD2 and CCM1: the cut of the keys
// found so far -- the team's best over those three (their indices precede
// VB2's) and the instance's slot -- often leaves only VB2 parameters up to
// a few thousand, which the unit then takes on the count table (S.vb2_mode 9;
// 10: none can matter; cluster_vb2, within kClusterVb2Terms lookups),
// flagging the instance's sums so (2) before any VB2 tile reads them.  The
// slot's key joins the team's maximum through thread 0
// of each CTA, so that every CTA of a cluster plans from the same key.  Only
// the cluster kernel's u-group units plan twice: in the prefix kernel the
// extra code, idle on the search-node step (whose first plan takes VB2), cost
// that step 1.5% (hard nodes gained 9%).
template <int MODE, class Team>
__device__ __forceinline__ void late_vb2_plan(const EvalArgs &A, const InstView &I, int64_t b,
                                           int64_t c, unsigned long long best, uint32_t L1,
                                           PrefixShared &S, unsigned long long *team, Team tm) {
  unsigned long long mine = best;
  if (threadIdx.x == 0) {
    const unsigned long long sk = *reinterpret_cast<const volatile unsigned long long *>(&A.keys[b]);
    mine = sk > mine ? sk : mine;
  }
  const unsigned long long kt = team_max_key(mine, S, team, tm);
  if (threadIdx.x == 0) {
    // vb2_cut's rule: a key before VB2's index wins ties, one after loses
    const uint32_t gv = flat_index(kVB2, 2, c);
    const int64_t cut =
        kt ? (int64_t)(kt >> 32) - ((0xFFFFFFFFu - (uint32_t)kt) < gv ? 0 : 1) : -1;
    int64_t kk = 0, lmax = 0;
    const int64_t vhi = A.vb2_hi != nullptr ? A.vb2_hi[b] : c;
    // the cut in place of L1 (MT in the bound: the caller's condition)
    const int mode = vb2_table_plan<MODE>(A, I, S, (uint32_t)max(cut, (int64_t)L1), vhi,
                                          kClusterVb2Terms, kk, lmax);
    S.vb2_mode = mode == 0 ? 0 : 8 + mode;  // 9, 10: planned late (9: evaluate)
    S.vb2_lmax = lmax;
  }
  __syncthreads();
}

// Evaluates the parameters of a built tile (prefix_tile; the cluster kernel):
// D's parameters [lam0, lam_end) -- after FS1's when with_fs1 (D = BJ1) --
// or the u group's members in umask, with the team's threads; returns the
// thread's best key.  The instance sums are in S.sums, the tables T0 (and T1)
// complete.  A team of several CTAs gathers FS1's sums in CTA 0 (fs1_gather),
// which forms FS1's bounds.
template <int MODE, int D, class Team, class Tab>
__device__ __forceinline__ unsigned long long prefix_evaluate(const EvalArgs &A, const InstView &I,
                                                              int64_t b, const Tab &T0,
                                                              const Tab &T1, int64_t c,
                                                              int64_t lam0, int64_t lam_end,
                                                              bool with_fs1, uint32_t umask,
                                                              PrefixShared &S, Team tm) {
  const uint32_t c32 = (uint32_t)c;
  // all below 2^31 on this path (prefix_handles); the sums S(l) below 2^32,
  // evaluated in wrapping 32-bit arithmetic
  PrefixEval x;
  x.c32 = c32;
  x.U = (uint32_t)((c - 1) / 2);
  x.n_big = (uint32_t)S.sums[1];
  x.n_half = (uint32_t)S.sums[2];
  x.n_full = (uint32_t)S.sums[3];
  x.sumw_big = (uint32_t)S.sums[4];
  x.sumw = (uint32_t)S.sums[5];
  x.TB = (uint32_t)S.sums[6];
  // L1 (MT's bound at l = 0) when MT is part of the bound, else no floor
  x.L1 = x.sumw / c32 + (x.sumw % c32 != 0u);
  x.B = (A.dff_off & 1u) ? 0u : x.L1;
  x.prune = A.prune && !(A.dff_off & 1u);
  x.best = 0ull;

  if (D == kBJ1 && with_fs1) {  // FS1 precedes BJ1 in paper order
    fs1_accumulate(T0, c, S, tm);
    __syncthreads();
    if constexpr (Team::kParts > 1) {
      fs1_gather(S, tm);
      tm.sync();
    }
    if (tm.part == 0u) fs1_finish(c, x, S);
  }
  if (D == kBJ1 && lam0 < lam_end) {  // FS1's lookups are done
    nn_to_d(T0, c32, tm);
    tm.sync();
  }
  if (D == kMT) eval_mt(T0, lam0, lam_end, c, x, tm);
  if (D == kRAD2) eval_rad2<false>(T0, T1, lam0, lam_end, c, x, tm);
  if (D == kCCM1 || D == kBJ1) {
    if constexpr (Team::kParts > 1) cluster_harmonic<D, false>(T0, lam0, lam_end, c, x, tm);
    else eval_harmonic<D, false>(T0, lam0, lam_end, c, x, S, tm);
  }
  if (D == kPrefixU) {
    // the members in paper order, so that each thread meets its parameters in
    // increasing flattened index
    auto member = [&](int d) { return ((umask >> d) & 1u) != 0u; };
    int64_t lo, hi;
    if (member(kMT)) {
      param_range(kMT, c, lo, hi);
      eval_mt(T0, lo, hi + 1, c, x, tm);
    }
    if (member(kRAD2)) {
      param_range(kRAD2, c, lo, hi);
      eval_rad2<true>(T0, T1, lo, hi + 1, c, x, tm);
    }
    if (member(kCCM1)) {
      param_range(kCCM1, c, lo, hi);
      if constexpr (Team::kParts > 1) cluster_harmonic<kCCM1, true>(T1, lo, hi + 1, c, x, tm);
      else eval_harmonic<kCCM1, true>(T1, lo, hi + 1, c, x, S, tm);
    }
    // VB2 stayed with its kernel at the first plan (cut L1): plan again with
    // the cut of the keys found so far (late_vb2_plan; cluster units)
    if constexpr (Team::kParts > 1) {
      if (S.vb2_mode == 0 && A.isums != nullptr && !A.verdict && A.prune && A.vb2_on &&
          !((A.dff_off >> kVB2) & 1u) && !(A.dff_off & 1u))
        late_vb2_plan<MODE>(A, I, b, c, x.best, x.L1, S, T1.team, tm);
    }
    if (S.vb2_mode == 1 || (Team::kParts > 1 && S.vb2_mode == 9)) {
      if constexpr (Team::kParts > 1) cluster_vb2(T1, c, x, S, S.vb2_lmax, tm);
      else eval_vb2_table(T1, c, x, S, S.vb2_lmax, tm);
    }
    if (Team::kParts > 1 && S.vb2_mode >= 9 && tm.part == 0u && threadIdx.x == 0) {
      __threadfence();  // VB2's keys are this tile's, folded with them
      A.isums[8 * b + 7] = 2;
    }
  }
  return x.best;
}

// Builds the table(s) of D (a DFF, or kPrefixU for the merged u group) for
// instance I -- one pass over the node's base items both accumulates its bin
// loads and histograms its unpacked items, a second pass histograms the bin
// loads -- and evaluates parameters [lam0, lam_end) (the u group: all of its
// members), after FS1's when with_fs1 (D = BJ1: the w-domain table; FS1's own
// tile is BJ1's with an empty range); returns the thread's best key.
template <int MODE, int D>
__device__ __forceinline__ unsigned long long prefix_tile(const EvalArgs &A, const InstView &I,
                                                          int64_t lam0, int64_t lam_end,
                                                          bool with_fs1, uint32_t umask,
                                                          int32_t *tab,
                                                          uint32_t *s_load, PrefixShared &S,
                                                          long long *isum_out, int64_t b) {
  const int tid = threadIdx.x;
  const int64_t c = I.c;
  const uint32_t c32 = (uint32_t)c;
  const uint32_t U = (uint32_t)((c - 1) / 2);
  const int nU = (int)U + 2, nW = (int)c + 2;
  int32_t *T0 = tab;       // E (MT, u group), N' (CCM1, RAD2), NN (BJ1)
  int32_t *T1 = tab + nU;  // Ns (RAD2), packed small/big counts (u group)
  const int nzero = (D == kBJ1) ? nW : ((D == kRAD2 || D == kPrefixU) ? 2 * nU : nU);
  {
    int4 *t4 = reinterpret_cast<int4 *>(tab);
    const int4 z = make_int4(0, 0, 0, 0);
    for (int i = tid; i < (nzero + 3) / 4; i += kPrefixNT) t4[i] = z;
  }
  const bool tr = MODE == kSrcNodes && bins_transformed(A);
  if (MODE == kSrcNodes)
    for (int64_t j = tid; j < I.k; j += kPrefixNT) s_load[j] = 0u;
  if (tr && tid == 0) S.minw = 0xFFFFFFFFu;
  if (tid < 8) S.sums[tid] = 0;
  if (D == kBJ1 && with_fs1 && tid < kFs1Params) {
    // FS1's parameters l = tid + 1 (l' = tid + 2)
    const uint32_t lp = (uint32_t)tid + 2u, cq = c32 / lp;
    S.fs1_cnt[tid] = 0u;
    S.fs1_dv[tid] = 0u;
    S.fs1_cq[tid] = cq;
    S.fs1_cr[tid] = c32 - cq * lp;
    S.fs1_mg[tid] = ((1u << 20) + lp - 1u) / lp;
  }
  __syncthreads();

  // ---- histogram the instance's reduced items ------------------------------------
  uint32_t ls[7] = {0, 0, 0, 0, 0, 0, 0};
  auto visit = [&](int64_t w) {
    if (w < 0 || w > c) {
      S.err = 1;
      return;
    }
    ls[5] += (uint32_t)w;
    if (D == kBJ1) {
      atomicAdd(&T0[w], 1);
      return;
    }
    if (w == 0) return;
    if (w == c) {
      ls[3]++;
    } else if (2 * w < c) {
      ls[0]++;
      atomicAdd(&T0[w], (D == kMT || D == kPrefixU) ? (int32_t)w : 1);
      if (D == kRAD2) atomicAdd(&T1[w], 1);
      if (D == kPrefixU) atomicAdd(reinterpret_cast<uint32_t *>(&T1[w]), 1u);
    } else if (2 * w > c) {
      const int64_t u = c - w;
      ls[1]++;
      ls[4] += (uint32_t)w;
      ls[6] += (uint32_t)u;
      atomicAdd(&T0[u], (D == kMT || D == kPrefixU) ? -(int32_t)u : -1);
      if (D == kPrefixU) atomicAdd(reinterpret_cast<uint32_t *>(&T1[u]), 1u << 16);
    } else {
      ls[2]++;
    }
  };
  if (MODE == kSrcNodes) {
    // the node's assignment and base sizes, 16 bytes per load where aligned
    for_items_vec<kPrefixNT, false>(I.a, I.w, I.n, [&](int64_t, int32_t a, int32_t w) {
      if (w < 0 || (int64_t)w > c || a < -1 || (int64_t)a >= I.k) {
        S.err = 1;
      } else if (a >= 0) {
        const uint32_t old = atomicAdd(&s_load[a], (uint32_t)w);
        if ((int64_t)old + w > c) S.err = 1;
      } else {
        visit(w);
        if (tr && w > 0) atomicMin(&S.minw, (uint32_t)w);
      }
    });
    __syncthreads();
    if (tr) {
      transform_bins<kPrefixNT>(A, b, I, s_load, S.minw, &S.err);
      __syncthreads();
    }
    for (int64_t j = tid; j < I.k; j += kPrefixNT) visit((int64_t)s_load[j]);
  } else if (MODE == kSrcRaggedI32) {
    // the instance's sizes, 16 bytes per load where aligned
    for_items_vec<kPrefixNT, true>(reinterpret_cast<const int32_t *>(A.sizes) + I.begin, nullptr, I.n,
                                   [&](int64_t, int32_t w, int32_t) { visit(w); });
  } else {
    const int64_t L = stream_len<MODE>(I);
    for (int64_t q = tid; q < L; q += kPrefixNT) {
      int64_t w = 0;
      fetch_item<MODE>(A, I, s_load, q, w);
      visit(w);
    }
  }
  // every count and sum is below 2^31 on this path: 32-bit warp reductions
#pragma unroll
  for (int e = 0; e < 7; ++e) {
    const uint32_t xs = __reduce_add_sync(0xFFFFFFFFu, ls[e]);
    if (lane_id() == 0 && xs != 0u) atomicAdd((unsigned long long *)&S.sums[e], (unsigned long long)xs);
  }
  __syncthreads();
  // VB2 on this tile (u group only; vb2_table_plan), then the class counts
  // and sums of the instance for the VB2 kernel's tile pruning (every tile
  // but BJ1's classifies the items), flagged 2 when VB2 is done here
  // (thread 0; the scans' barriers publish S.vb2_* before they are read)
  if (threadIdx.x == 0) {
    int mode = 0;
    int64_t kk = 0, lmax = 0;
    if (D == kPrefixU && !S.err) {
      const uint32_t sw32 = (uint32_t)S.sums[5];
      const int64_t vhi = A.vb2_hi != nullptr ? A.vb2_hi[b] : c;
      mode = vb2_table_plan<MODE>(A, I, S, sw32 / c32 + (sw32 % c32 != 0u), vhi, kVb2TableTerms,
                                  kk, lmax);
    }
    S.vb2_mode = mode;
    S.vb2_kk = kk;
    S.vb2_lmax = lmax;
    if (D != kBJ1 && isum_out != nullptr && !S.err) {
#pragma unroll
      for (int e = 0; e < 6; ++e) isum_out[e] = S.sums[e];
      __threadfence();
      isum_out[7] = mode != 0 ? 2 : 1;
    }
  }
  if (D == kBJ1) {
    suffix_scan<true>(T0, nW, S);
  } else {
    suffix_scan<false>(T0, nU, S);
    if (D == kRAD2) suffix_scan<false>(T1, nU, S);
    if (D == kPrefixU) packed_count_scan(reinterpret_cast<uint32_t *>(T1), nU, S);
  }
  if (S.err) return 0ull;

  return prefix_evaluate<MODE, D>(A, I, b, LocalTab{T0}, LocalTab{T1}, c, lam0, lam_end, with_fs1,
                                  umask, S, CtaTeam{0u});
}

// Persistent kernel over the prefix tile table (instance, DFF in {MT, RAD2,
// FS1, CCM1, BJ1} routed here by prefix_handles or the merged u group, A.plpt
// consecutive lambdas -- all of them when the tables are in the global
// scratch; FS1 with BJ1's first tile when prefix_w_merged).  Tables of a
// cluster's size (prefix_home 3) are the cluster kernel's (bp_lb_cluster.cuh).
template <int MODE>
__global__ void __launch_bounds__(kPrefixNT, 4) prefix_kernel(EvalArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PrefixShared S;
  __shared__ TileCursor cur;
  int32_t *stab = reinterpret_cast<int32_t *>(smem_raw);
  uint32_t *s_load = reinterpret_cast<uint32_t *>(smem_raw + kPrefixSmemBytes);

  pdl_wait();
  pdl_release();
  const int64_t total = A.ptile_start ? A.ptile_start[A.B] : A.single_ptiles;
  if (threadIdx.x == 0) S.rc_c = -1;  // no routing cached yet
  tile_first(A.ptile_start, A.B, total, A.pwork, cur);
  while (cur.tile < total) {
    const int64_t t = cur.tile, b = cur.inst;
    const unsigned long long next = tile_claim(A.pwork);
    const InstView I = resolve_instance<MODE>(A, b);
    const int64_t t0 = A.ptile_start ? A.ptile_start[b] : 0;
    const int64_t ntiles = instance_tiles(A, b);
    // which DFF (or the merged u group) and lambdas, tables in shared memory
    // or in this CTA's slice of the global scratch: decoded by thread 0
    if (threadIdx.x == 0) {
      int64_t rem = t - t0;
      int d = 0;
      const int64_t sb = sum_bound<MODE>(I);
      const int rk = route_class(I.c, sb);
      if (I.c != S.rc_c || rk != S.rc_k) {  // route this instance (tile counts as route_tiles)
        const bool merged = prefix_u_merged(I.c, sb, A.prefix_on, A.vb2_on, A.dff_off, A.plpt);
        const bool wmerged = prefix_w_merged(I.c, sb, A.prefix_on, A.vb2_on, A.dff_off);
        int umask = 0;
        for (int e = 0; e < kNumDff; ++e) {
          const bool pre = dff_kernel(e, I.c, sb, A.prefix_on, A.vb2_on, A.dff_off) == kRoutePrefix;
          const bool member = merged && (e == kMT || e == kRAD2 || e == kCCM1);
          if (member && param_count(e, I.c) > 0 && pre) umask |= 1 << e;
          S.rc_home[e] = prefix_home(e, I.c, sb, A.prefix_on);
          // units whose tables are a cluster's go to the cluster kernel
          S.rc_nt[e] = (pre && !member && !(wmerged && e == kFS1) && S.rc_home[e] != 3)
                           ? (int)prefix_dff_tiles(e, I.c, sb, A.prefix_on, A.plpt)
                           : 0;
        }
        S.rc_merged = merged && prefix_u_home(I.c, A.prefix_on) != 3;
        S.rc_wmerged = wmerged;
        S.rc_umask = umask;
        S.rc_uhome = prefix_u_home(I.c, A.prefix_on);
        S.rc_c = I.c;
        S.rc_k = rk;
      }
      const bool merged = S.rc_merged != 0, wmerged = S.rc_wmerged != 0;
      if (merged && rem == 0) {
        d = kPrefixU;
      } else {
        if (merged) rem -= 1;  // the u group's tile comes first
        for (d = 0; d < kNumDff; ++d) {
          const int64_t nt = S.rc_nt[d];
          if (rem < nt) break;
          rem -= nt;
        }
      }
      const int home = (d == kPrefixU) ? S.rc_uhome : (d < kNumDff ? S.rc_home[d] : 0);
      int64_t lo_d = 0, hi_d = -1;
      if (d != kPrefixU && d != kFS1) param_range(d, I.c, lo_d, hi_d);
      const int64_t lpt = (home == 2) ? hi_d - lo_d + 1 : A.plpt;  // global tables: one tile
      const int64_t lam0 = lo_d + rem * lpt;
      const int umask = d == kPrefixU ? S.rc_umask : 0;
      S.dec_d = d;
      S.dec_home = home;
      // FS1 on BJ1's table: on its own tile (empty BJ1 range) or BJ1's first
      S.dec_fs1 = (d == kFS1 || (wmerged && d == kBJ1 && rem == 0)) ? 1 : 0;
      S.dec_umask = umask;
      S.dec_lam0 = lam0;
      S.dec_lam_end = min(hi_d + 1, lam0 + lpt);
      S.err = 0;
      S.skip = (A.verdict && slot_decided(&A.keys[b], I.k)) ? 1 : 0;
    }
    __syncthreads();
    const int d = S.dec_d, home = S.dec_home;
    const bool with_fs1 = S.dec_fs1 != 0;
    const int64_t lam0 = S.dec_lam0, lam_end = S.dec_lam_end;
    const uint32_t umask = (uint32_t)S.dec_umask;
    int32_t *gtab = A.gscratch + (size_t)blockIdx.x * (size_t)kGlobalTableInts;
    long long *isum = A.isums != nullptr ? A.isums + 8 * b : nullptr;
    unsigned long long best = 0ull;
    // one instantiation per table space, so that shared-memory tables are
    // accessed with shared-memory instructions
    if (!S.skip && home != 2) {
      if (d == kPrefixU) best = prefix_tile<MODE, kPrefixU>(A, I, lam0, lam_end, false, umask, stab, s_load, S, isum, b);
      else if (d == kMT) best = prefix_tile<MODE, kMT>(A, I, lam0, lam_end, false, umask, stab, s_load, S, isum, b);
      else if (d == kRAD2) best = prefix_tile<MODE, kRAD2>(A, I, lam0, lam_end, false, umask, stab, s_load, S, isum, b);
      else if (d == kCCM1) best = prefix_tile<MODE, kCCM1>(A, I, lam0, lam_end, false, umask, stab, s_load, S, isum, b);
      else best = prefix_tile<MODE, kBJ1>(A, I, lam0, lam_end, with_fs1, 0u, stab, s_load, S, nullptr, b);
    } else if (!S.skip) {
      if (d == kPrefixU) best = prefix_tile<MODE, kPrefixU>(A, I, lam0, lam_end, false, umask, gtab, s_load, S, isum, b);
      else if (d == kMT) best = prefix_tile<MODE, kMT>(A, I, lam0, lam_end, false, umask, gtab, s_load, S, isum, b);
      else if (d == kRAD2) best = prefix_tile<MODE, kRAD2>(A, I, lam0, lam_end, false, umask, gtab, s_load, S, isum, b);
      else if (d == kCCM1) best = prefix_tile<MODE, kCCM1>(A, I, lam0, lam_end, false, umask, gtab, s_load, S, isum, b);
      else best = prefix_tile<MODE, kBJ1>(A, I, lam0, lam_end, with_fs1, 0u, gtab, s_load, S, nullptr, b);
    }
    __syncthreads();
    fold_and_finalize<kPrefixNT>(A, b, best, S.err != 0, ntiles, I, S.warp_key);
    if (!A.pwork) break;
    tile_publish(A.ptile_start, A.B, total, next, cur);
  }
}

}  // namespace bplb
