// bp_lb_cluster.cuh -- prefix-count evaluation (bp_lb_prefix.cuh) of tables
// too large for one CTA's shared memory, spread over a thread-block cluster.
//
// A unit is what the prefix kernel would give one CTA with its tables in the
// global scratch: an instance's merged u group (MT, RAD2, CCM1), one of MT,
// RAD2 or CCM1 alone, BJ1 with FS1, or FS1 alone, each over its whole
// parameter range (prefix_home 3; route_tiles(kRouteCluster) counts them per
// instance).  A cluster of kClusterCtas CTAs takes a unit.  Its tables -- the
// prefix kernel's, entries 0 .. nzero - 1 -- are cut into slices of
// kSliceInts entries, slice r in CTA r's shared memory, and every CTA reads
// and writes any entry through distributed shared memory (ClusterTab).
// Phases, separated by cluster barriers:
//   1. each CTA zeroes its slice (and for a search node computes the node's
//      bin loads itself, from all of its items);
//   2. histogram: each CTA visits its share of the reduced items, adding into
//      the owning slices (red.shared::cluster); the instance sums and the
//      error flag gather in CTA 0 and are read back by every CTA;
//   3. suffix scans: each CTA scans its part of each table from the carries of
//      the parts above it (their totals gather in CTA 0);
//   4. lookups: prefix_evaluate with the cluster as one team -- the
//      parameters dealt over its kClusterCtas x kPrefixNT threads as the
//      prefix kernel deals them over one CTA's;
//   5. each CTA's best key goes to CTA 0, which folds the unit into the
//      instance's result slot and takes its finished-tile ticket.
// Every branch around a cluster barrier depends only on values that every CTA
// of the cluster holds alike (the unit, the instance, the gathered error
// flag), so that all of them arrive at the same barriers.
#pragma once

#include "bp_lb_prefix.cuh"

namespace bplb {

constexpr int64_t kSliceBytes = 4 * kSliceInts;
using ClusterTeam = Team<kClusterCtas>;

// Gathering points in CTA 0 of the cluster (the other CTAs reach them through
// distributed shared memory), and each CTA's copy of the scan totals.
struct ClusterShared {
  unsigned long long next;               // the unit the cluster takes next
  int err;                               // OR of the CTAs' error flags
  long long sums[8];                     // the instance sums (PrefixShared::sums)
  uint32_t tot[kClusterCtas][3];         // per CTA: H, M of its part of T0, H of T1's
  uint32_t ltot[kClusterCtas][3];        // this CTA's copy of tot
  unsigned long long key[kClusterCtas];   // per CTA: its best key
  unsigned long long team[kClusterCtas];  // per CTA: its best key so far (late_vb2_plan)
};

// The part [a, e) (slice-local entries) of this CTA's slice that cluster
// entries [lo, hi) cover; a == e when none.
__device__ __forceinline__ void slice_part(uint32_t rank, uint32_t lo, uint32_t hi, uint32_t &a,
                                           uint32_t &e) {
  const uint32_t s0 = rank << kSliceShift, s1 = s0 + (uint32_t)kSliceInts;
  const uint32_t x0 = max(lo, s0), x1 = min(hi, s1);
  a = min(x0, s1) - s0;
  e = x1 > x0 ? x1 - s0 : a;
}

// Totals of a[0 .. n) over the CTA: H = sum a[i] and (TWICE) M = sum (i + 1)
// a[i], in wrapping 32-bit arithmetic like suffix_scan.  Thread 0 gets them.
template <bool TWICE>
__device__ __forceinline__ void part_totals(const int32_t *a, int n, PrefixShared &S, uint32_t &H,
                                            uint32_t &M) {
  const int per = ((n + kPrefixNT - 1) / kPrefixNT) | 1;
  const int s0 = min(n, (int)threadIdx.x * per), s1 = min(n, s0 + per);
  uint32_t h = 0, m = 0;
  for (int i = s0; i < s1; ++i) {
    const uint32_t v = (uint32_t)a[i];
    h += v;
    if (TWICE) m += v * (uint32_t)(i + 1);
  }
  h = warp_sum(h);
  if (TWICE) m = warp_sum(m);
  const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
  if (lane == 0) {
    S.wtot[0][warp] = h;
    S.wtot[1][warp] = m;
  }
  __syncthreads();
  H = 0;
  M = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kPrefixWarps; ++w) {
      H += S.wtot[0][w];
      M += S.wtot[1][w];
    }
  __syncthreads();
}

// One unit (file comment) of instance I; D is kPrefixU, kMT, kRAD2, kCCM1 or
// kBJ1 (FS1 alone: BJ1's tables with an empty range and with_fs1).  Returns
// the thread's best key (0 after an error, which S.err then holds alike in
// every CTA).
template <int MODE, int D>
__device__ __forceinline__ unsigned long long cluster_unit(const EvalArgs &A, const InstView &I,
                                                           int64_t b, int64_t lam0,
                                                           int64_t lam_end, bool with_fs1,
                                                           uint32_t umask, int32_t *slice,
                                                           uint32_t *s_load, PrefixShared &S,
                                                           ClusterShared &C, ClusterTeam tm) {
  const int tid = threadIdx.x;
  const uint32_t rank = tm.part;
  const int64_t c = I.c;
  const uint32_t c32 = (uint32_t)c;
  const uint32_t U = (uint32_t)((c - 1) / 2);
  const uint32_t nU = U + 2u, nW = c32 + 2u;
  uint32_t *acc = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(slice) + kSliceBytes);
  const ClusterTab T0{smem_addr(slice), 0u, slice, acc, C.team};
  const ClusterTab T1 = T0.at(nU);  // Ns (RAD2), packed small/big counts (u group)
  const uint32_t nT0 = (D == kBJ1) ? nW : nU;
  const uint32_t nzero = (D == kRAD2 || D == kPrefixU) ? 2u * nU : nT0;

  // ---- 1. zero this CTA's slice; per-CTA state -------------------------------------
  {
    uint32_t a, e;
    slice_part(rank, 0u, nzero, a, e);
    int4 *t4 = reinterpret_cast<int4 *>(slice);
    const int4 z = make_int4(0, 0, 0, 0);
    for (uint32_t i = tid; i < (e + 3u) / 4u; i += kPrefixNT) t4[i] = z;
  }
  const bool tr = MODE == kSrcNodes && bins_transformed(A);
  if (MODE == kSrcNodes)
    for (int64_t j = tid; j < I.k; j += kPrefixNT) s_load[j] = 0u;
  if (tr && tid == 0) S.minw = 0xFFFFFFFFu;
  if (tid < 8) S.sums[tid] = 0;
  if (tid == 0) S.err = 0;
  if (rank == 0u) {
    if (tid < 8) C.sums[tid] = 0;
    if (tid == 0) C.err = 0;
  }
  for (uint32_t i = tid; i < kOwnPerCta; i += kPrefixNT) acc[i] = 0u;  // cluster_harmonic's
  if (D == kBJ1 && with_fs1 && tid < kFs1Params) {
    // FS1's parameters l = tid + 1 (l' = tid + 2), in every CTA
    const uint32_t lp = (uint32_t)tid + 2u, cq = c32 / lp;
    S.fs1_cnt[tid] = 0u;
    S.fs1_dv[tid] = 0u;
    S.fs1_cq[tid] = cq;
    S.fs1_cr[tid] = c32 - cq * lp;
    S.fs1_mg[tid] = ((1u << 20) + lp - 1u) / lp;
  }
  cluster_barrier();  // every slice zeroed before any CTA adds into it

  // ---- 2. histogram of this CTA's share of the reduced items ---------------------------
  uint32_t ls[7] = {0, 0, 0, 0, 0, 0, 0};
  auto visit = [&](int64_t w) {
    if (w < 0 || w > c) {
      S.err = 1;
      return;
    }
    ls[5] += (uint32_t)w;
    if (D == kBJ1) {
      T0.add((uint32_t)w, 1);
      return;
    }
    if (w == 0) return;
    if (w == c) {
      ls[3]++;
    } else if (2 * w < c) {
      ls[0]++;
      T0.add((uint32_t)w, (D == kMT || D == kPrefixU) ? (int32_t)w : 1);
      if (D == kRAD2 || D == kPrefixU) T1.add((uint32_t)w, 1);
    } else if (2 * w > c) {
      const int64_t u = c - w;
      ls[1]++;
      ls[4] += (uint32_t)w;
      ls[6] += (uint32_t)u;
      T0.add((uint32_t)u, (D == kMT || D == kPrefixU) ? -(int32_t)u : -1);
      if (D == kPrefixU) T1.add((uint32_t)u, 1 << 16);
    } else {
      ls[2]++;
    }
  };
  if (MODE == kSrcNodes) {
    // every CTA reads the whole node (the bin loads need all of it) and
    // visits the unpacked items i with i mod kClusterCtas == rank, then its
    // share of the bins
    for_items_vec<kPrefixNT, false>(I.a, I.w, I.n, [&](int64_t i, int32_t a, int32_t w) {
      if (w < 0 || (int64_t)w > c || a < -1 || (int64_t)a >= I.k) {
        S.err = 1;
      } else if (a >= 0) {
        const uint32_t old = atomicAdd(&s_load[a], (uint32_t)w);
        if ((int64_t)old + w > c) S.err = 1;
      } else {
        if (((uint32_t)i & (uint32_t)(kClusterCtas - 1)) == rank) visit(w);
        if (tr && w > 0) atomicMin(&S.minw, (uint32_t)w);
      }
    });
    __syncthreads();
    if (tr) {
      transform_bins<kPrefixNT>(A, b, I, s_load, S.minw, &S.err);
      __syncthreads();
    }
    for (int64_t j = tm.tid(); j < I.k; j += ClusterTeam::kThreads) visit((int64_t)s_load[j]);
  } else if (MODE == kSrcRaggedI32) {
    for_items_vec<kPrefixNT, true, kClusterCtas>(
        reinterpret_cast<const int32_t *>(A.sizes) + I.begin, nullptr, I.n,
        [&](int64_t, int32_t w, int32_t) { visit(w); }, rank);
  } else {
    const int64_t L = stream_len<MODE>(I);
    for (int64_t q = tm.tid(); q < L; q += ClusterTeam::kThreads) {
      int64_t w = 0;
      fetch_item<MODE>(A, I, s_load, q, w);
      visit(w);
    }
  }
  // the counts and sums of this CTA's share (below 2^31 on this path), then
  // into CTA 0
#pragma unroll
  for (int e = 0; e < 7; ++e) {
    const uint32_t xs = __reduce_add_sync(0xFFFFFFFFu, ls[e]);
    if (lane_id() == 0 && xs != 0u) atomicAdd((unsigned long long *)&S.sums[e], (unsigned long long)xs);
  }
  __syncthreads();
  if (tid < 7 && S.sums[tid] != 0)
    dsm_red_add64(cluster_map(smem_addr(&C.sums[tid]), 0), (unsigned long long)S.sums[tid]);
  if (tid == 0 && S.err) dsm_red_or(cluster_map(smem_addr(&C.err), 0), 1u);
  cluster_barrier();  // histogram, sums and error flag complete
  if (tid < 8) S.sums[tid] = (long long)dsm_ld64(cluster_map(smem_addr(&C.sums[tid]), 0));
  if (tid == 0) S.err = dsm_ld(cluster_map(smem_addr(&C.err), 0));
  __syncthreads();
  // VB2 on the u group (vb2_table_plan, in every CTA alike) and the instance
  // sums for the other kernels (CTA 0), as in prefix_tile
  if (tid == 0) {
    int mode = 0;
    int64_t kk = 0, lmax = 0;
    if (D == kPrefixU && !S.err) {
      const uint32_t sw32 = (uint32_t)S.sums[5];
      const int64_t vhi = A.vb2_hi != nullptr ? A.vb2_hi[b] : c;
      mode = vb2_table_plan<MODE>(A, I, S, sw32 / c32 + (sw32 % c32 != 0u), vhi,
                                  kClusterCtas * kVb2TableTerms, kk, lmax);
    }
    S.vb2_mode = mode;
    S.vb2_kk = kk;
    S.vb2_lmax = lmax;
    long long *isum_out = A.isums != nullptr ? A.isums + 8 * b : nullptr;
    if (rank == 0u && D != kBJ1 && isum_out != nullptr && !S.err) {
#pragma unroll
      for (int e = 0; e < 6; ++e) isum_out[e] = S.sums[e];
      __threadfence();
      isum_out[7] = mode != 0 ? 2 : 1;
    }
  }
  __syncthreads();
  if (S.err) return 0ull;  // alike in every CTA

  // ---- 3. suffix scans of this CTA's parts, from the parts above --------------------------
  constexpr bool TWO = D == kRAD2 || D == kPrefixU;
  uint32_t a0, e0, a1 = 0u, e1 = 0u;
  slice_part(rank, 0u, nT0, a0, e0);
  if (TWO) slice_part(rank, nU, 2u * nU, a1, e1);
  uint32_t H0, M0, H1 = 0u, M1;
  part_totals<D == kBJ1>(slice + a0, (int)(e0 - a0), S, H0, M0);
  if (TWO) part_totals<false>(slice + a1, (int)(e1 - a1), S, H1, M1);
  if (tid == 0) {
    dsm_st(cluster_map(smem_addr(&C.tot[rank][0]), 0), (int32_t)H0);
    dsm_st(cluster_map(smem_addr(&C.tot[rank][1]), 0), (int32_t)M0);
    dsm_st(cluster_map(smem_addr(&C.tot[rank][2]), 0), (int32_t)H1);
  }
  cluster_barrier();  // every part's totals in CTA 0
  if (tid < 3 * kClusterCtas)
    (&C.ltot[0][0])[tid] = (uint32_t)dsm_ld(cluster_map(smem_addr(&(&C.tot[0][0])[tid]), 0));
  __syncthreads();
  // carries from the parts above: N = sum of their entries, NN = sum over
  // them of the once-scanned entries (M of a part plus its length times the
  // count above it)
  uint32_t n0 = 0u, nn0 = 0u, n1 = 0u;
  for (uint32_t r = kClusterCtas - 1; r > rank; --r) {
    uint32_t pa, pe;
    slice_part(r, 0u, nT0, pa, pe);
    nn0 += C.ltot[r][1] + (pe - pa) * n0;
    n0 += C.ltot[r][0];
    n1 += C.ltot[r][2];
  }
  if (D == kBJ1) {
    suffix_scan<true>(slice + a0, (int)(e0 - a0), S, n0, nn0);
  } else {
    suffix_scan<false>(slice + a0, (int)(e0 - a0), S, n0, 0u);
    if (D == kRAD2) suffix_scan<false>(slice + a1, (int)(e1 - a1), S, n1, 0u);
    if (D == kPrefixU)
      packed_count_scan(reinterpret_cast<uint32_t *>(slice + a1), (int)(e1 - a1), S, n1);
  }
  cluster_barrier();  // the tables complete

  // ---- 4. lookups ------------------------------------------------------------------
  return prefix_evaluate<MODE, D>(A, I, b, T0, T1, c, lam0, lam_end, with_fs1, umask, S, tm);
}

// The unit of the cluster kernel's table entry t - t0 of instance I (the
// order route_tiles(kRouteCluster) counts them in); thread 0.
template <int MODE>
__device__ __forceinline__ void cluster_decode(const EvalArgs &A, const InstView &I, int64_t rem,
                                               PrefixShared &S) {
  const int64_t c = I.c;
  const int64_t sb = sum_bound<MODE>(I);
  const bool merged = prefix_u_merged(c, sb, A.prefix_on, A.vb2_on, A.dff_off, A.plpt);
  const bool wmerged = prefix_w_merged(c, sb, A.prefix_on, A.vb2_on, A.dff_off);
  const bool ucl = merged && prefix_u_home(c, A.prefix_on) == 3;
  int d = kPrefixU, umask = 0;
  if (ucl) {
    for (int e = 0; e < kNumDff; ++e)
      if ((e == kMT || e == kRAD2 || e == kCCM1) && param_count(e, c) > 0 &&
          dff_kernel(e, c, sb, A.prefix_on, A.vb2_on, A.dff_off) == kRoutePrefix)
        umask |= 1 << e;
  }
  if (!(ucl && rem == 0)) {
    if (ucl) rem -= 1;
    for (d = 0; d < kNumDff; ++d) {
      if (merged && (d == kMT || d == kRAD2 || d == kCCM1)) continue;
      if (wmerged && d == kFS1) continue;
      if (dff_kernel(d, c, sb, A.prefix_on, A.vb2_on, A.dff_off) != kRoutePrefix ||
          prefix_home(d, c, sb, A.prefix_on) != 3 || param_count(d, c) == 0)
        continue;
      if (rem == 0) break;
      --rem;
    }
  }
  int64_t lo_d = 0, hi_d = -1;
  if (d < kNumDff && d != kFS1) param_range(d, c, lo_d, hi_d);
  S.dec_d = d;  // kNumDff: no such unit (an inconsistent table; reported as an error)
  S.dec_fs1 = (d == kFS1 || (wmerged && d == kBJ1)) ? 1 : 0;
  S.dec_umask = umask;
  S.dec_lam0 = lo_d;
  S.dec_lam_end = hi_d + 1;
}

// Persistent over the cluster unit table (A.ctile_start; A.cwork counts the
// units claimed), or one unit per cluster (single instance, A.cwork null).
template <int MODE>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kPrefixNT, 3)
    cluster_kernel(EvalArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PrefixShared S;
  __shared__ ClusterShared C;
  __shared__ unsigned long long s_t;
  __shared__ long long s_b;
  int32_t *slice = reinterpret_cast<int32_t *>(smem_raw);
  // dynamic shared memory: the table slice, cluster_harmonic's accumulators,
  // the bin loads (search nodes)
  uint32_t *s_load = reinterpret_cast<uint32_t *>(smem_raw + kSliceBytes + kOwnBytes);
  const int tid = threadIdx.x;
  const ClusterTeam tm{cluster_rank()};
  const unsigned long long total =
      (unsigned long long)(A.ctile_start ? A.ctile_start[A.B] : A.single_ctiles);
  const bool persistent = A.cwork != nullptr;
  if (tm.part == 0u && tid == 0)
    C.next = persistent ? (total > 0ull ? atomicAdd(A.cwork, 1ull) : ~0ull)
                        : (unsigned long long)(blockIdx.x / kClusterCtas);
  for (;;) {
    cluster_barrier();  // the unit claimed; no CTA reads the last unit's tables
    if (tid == 0) s_t = dsm_ld64(cluster_map(smem_addr(&C.next), 0));
    __syncthreads();
    const unsigned long long t = s_t;
    if (t >= total) break;  // alike in every CTA
    if (tid < 32) {
      int64_t b = 0;
      if (A.ctile_start) b = warp_find_instance(A.ctile_start, A.B, (int64_t)t);
      if (tid == 0) {
        s_b = b;
        const InstView I = resolve_instance<MODE>(A, b);
        cluster_decode<MODE>(A, I, (int64_t)t - (A.ctile_start ? A.ctile_start[b] : 0), S);
      }
    }
    __syncthreads();
    const int64_t b = s_b;
    const InstView I = resolve_instance<MODE>(A, b);
    const int d = S.dec_d;
    const bool with_fs1 = S.dec_fs1 != 0;
    const int64_t lam0 = S.dec_lam0, lam_end = S.dec_lam_end;
    const uint32_t umask = (uint32_t)S.dec_umask;
    unsigned long long best = 0ull;
    bool bad = false;
    if (d == kPrefixU)
      best = cluster_unit<MODE, kPrefixU>(A, I, b, lam0, lam_end, false, umask, slice, s_load, S, C, tm);
    else if (d == kMT)
      best = cluster_unit<MODE, kMT>(A, I, b, lam0, lam_end, false, 0u, slice, s_load, S, C, tm);
    else if (d == kRAD2)
      best = cluster_unit<MODE, kRAD2>(A, I, b, lam0, lam_end, false, 0u, slice, s_load, S, C, tm);
    else if (d == kCCM1)
      best = cluster_unit<MODE, kCCM1>(A, I, b, lam0, lam_end, false, 0u, slice, s_load, S, C, tm);
    else if (d == kBJ1 || d == kFS1)
      best = cluster_unit<MODE, kBJ1>(A, I, b, lam0, lam_end, with_fs1, 0u, slice, s_load, S, C, tm);
    else
      bad = true;
    // ---- 5. the cluster's best key into CTA 0, which folds the unit ---------------
    best = warp_max_u64(best);
    if (lane_id() == 0) S.warp_key[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
      unsigned long long m = 0ull;
      for (int w = 0; w < kPrefixWarps; ++w) m = S.warp_key[w] > m ? S.warp_key[w] : m;
      dsm_st64(cluster_map(smem_addr(&C.key[tm.part]), 0), m);
    }
    cluster_barrier();  // every CTA's key in CTA 0
    if (tm.part == 0u) {
      const unsigned long long kb = tid < kClusterCtas ? C.key[tid] : 0ull;
      fold_and_finalize<kPrefixNT>(A, b, kb, bad || S.err != 0, instance_tiles(A, b), I,
                                   S.warp_key);
      if (tid == 0) C.next = persistent ? atomicAdd(A.cwork, 1ull) : ~0ull;
    }
  }
  cluster_barrier();  // no CTA leaves while another may still read its shared memory
}

}  // namespace bplb
