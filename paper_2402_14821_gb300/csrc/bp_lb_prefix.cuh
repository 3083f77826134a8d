// bp_lb_prefix.cuh -- prefix-count evaluation of MT, CCM1 and BJ1.
//
// Same bounds as the direct evaluators (bit-exact), asymptotically less work:
// per tile the instance's items are histogrammed by value in shared memory and
// scanned, after which each parameter needs O(1) (MT), O(U / l) (CCM1) or
// O(c / l) (BJ1) table lookups instead of one evaluation per item:
//
//   MT:   sum_small u [u >= l] + sum_big u [u < l] = E(l) + TB, with
//         E(x) = sum over values y >= x of (small sum at y - big sum at y)
//         and TB the total of the big u;
//   CCM1: sum_small floor(u / l) - sum_big floor(u / l) = sum_{j >= 1} N(j l),
//         with N(x) = #small[u >= x] - #big[u >= x], since floor(u / l) counts
//         the multiples j l <= u;
//   BJ1:  sum_w (cm q + min(rho, cm)) over the blocks [j l, j l + l) of the
//         value range (q = j inside block j):
//           cm * sum_{j >= 1} #[w >= j l]
//         + sum_j ( sum_{w in [jl, jl + cm)} (w - j l) + cm #[w in [jl + cm, jl + l)] ),
//         read from the prefix count C(x) = #[w < x] and prefix sum
//         Sm(x) = sum_{w < x} w.
// (u, the small/big classes, cm = c mod l and the sums assembled from these
// accumulators are those of bp_lb_core.cuh.)  VB2, RAD2 and FS1 stay on the
// direct kernel.
#pragma once

#include "bp_lb_kernels.cuh"

namespace bplb {

constexpr int kPrefixNT = 256;
// Parameters needing more lookups than this are "heavy": the whole CTA
// shares their lookups; the others take one thread each.
constexpr int kHeavyBlocks = 256;
constexpr int kMaxHeavy = 256;

struct PrefixShared {
  int err;
  int pad_;
  unsigned long long warp_key[kPrefixNT / 32];
  long long sums[8];  // n_small, n_big, n_half, n_full, sumw_big, sumw, total big u, total count
  int64_t seg[kPrefixNT];
  unsigned long long heavy_acc[kMaxHeavy];  // two's-complement partial sums of heavy parameters
};

// Shared-memory array lengths (entries) of the prefix tables.
BPLB_HD int64_t prefix_u_len(int64_t c) { return (c - 1) / 2 + 2; }   // u in [0, (c-1)/2] + 0-sentinel
BPLB_HD int64_t prefix_w_len(int64_t c) { return c + 2; }             // x in [0, c + 1]

// In-place block-wide scan of a[0 .. n): inclusive suffix sums (SUFFIX) or
// exclusive prefix sums.  Each thread scans one contiguous segment serially;
// the segment totals are scanned with warp shuffles (every warp its 32
// totals, then warp 0 the warp totals).
template <bool SUFFIX>
__device__ void block_scan_i32(int32_t *a, int n, int64_t *seg) {
  const int tid = threadIdx.x;
  const int per = (n + kPrefixNT - 1) / kPrefixNT;
  const int s0 = min(n, tid * per), s1 = min(n, s0 + per);
  int64_t tot = 0;
  for (int i = s0; i < s1; ++i) tot += a[SUFFIX ? n - 1 - i : i];
  // inclusive scan of the totals within the warp
  int64_t x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if ((int)lane_id() >= o) x += y;
  }
  if (lane_id() == 31) seg[tid >> 5] = x;
  __syncthreads();
  if (tid < 32) {
    int64_t wv = tid < kPrefixNT / 32 ? seg[tid] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, wv, o);
      if (tid >= o) wv += y;
    }
    if (tid < kPrefixNT / 32) seg[32 + tid] = wv;  // inclusive warp prefix
  }
  __syncthreads();
  int64_t run = x - tot + ((tid >> 5) ? seg[32 + (tid >> 5) - 1] : 0);  // exclusive
  for (int i = s0; i < s1; ++i) {
    const int idx = SUFFIX ? n - 1 - i : i;
    const int64_t v = a[idx];
    if (SUFFIX) {
      run += v;
      a[idx] = (int32_t)run;
    } else {
      a[idx] = (int32_t)run;
      run += v;
    }
  }
  __syncthreads();
}

// Bin loads of a search node into s_load (shared with the direct kernel's
// staging); sets *err for a bad assignment or an overfull bin.
template <int NT, int MODE>
__device__ __forceinline__ void node_loads(const InstView &I, uint32_t *s_load, int *err) {
  if (MODE == kSrcNodes) {
    for (int64_t j = threadIdx.x; j < I.k; j += NT) s_load[j] = 0u;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < I.n; i += NT) {
      const int32_t a = I.a[i];
      const int32_t w = I.w[i];
      if (w < 0 || (int64_t)w > I.c || a < -1 || (int64_t)a >= I.k) {
        *err = 1;
      } else if (a >= 0) {
        const uint32_t old = atomicAdd(&s_load[a], (uint32_t)w);
        if ((int64_t)old + w > I.c) *err = 1;
      }
    }
  }
}

// One parameter's accumulator, lanes `lane` (stride `stride`) of its blocks.
template <int D>
__device__ __forceinline__ int64_t prefix_acc(const int32_t *T0, const int32_t *T1, int64_t c,
                                              int64_t l, int lane, int stride, int64_t R,
                                              int64_t TB) {
  int64_t acc = 0;
  if (D == kMT) {
    if (lane == 0) {
      const int64_t U1 = prefix_u_len(c) - 1;  // sentinel index
      acc = (int64_t)T0[l < U1 ? l : U1] + TB;
    }
  } else if (D == kCCM1) {
    // indices < 2^31 (c <= 2^30): 32-bit loop arithmetic
    const uint32_t U = (uint32_t)(prefix_u_len(c) - 2), l32 = (uint32_t)l;
    const uint32_t step = (uint32_t)stride * l32;
    int32_t a32 = 0;  // partial sums of at most U / l terms of |N| <= r: 32 bits suffice
    for (uint32_t x = (1u + (uint32_t)lane) * l32; x <= U; x += step) a32 += T0[x];
    acc = a32;
  } else {  // BJ1: T0 = C (prefix count), T1 = Sm (prefix sum)
    const uint32_t c32 = (uint32_t)c, l32 = (uint32_t)l;
    const uint32_t cm = c32 % l32;
    const uint32_t top = c32 + 1u;
    const uint32_t step = (uint32_t)stride * l32;
    int64_t nq = 0;  // sum over blocks j >= 1 of #[w >= j l]
    for (uint32_t a = (uint32_t)lane * l32; a <= c32; a += step) {
      const uint32_t b1 = min(a + cm, top), b2 = min(a + l32, top);
      const int32_t Ca = T0[a], Cb1 = T0[b1], Cb2 = T0[b2];
      acc += (int64_t)(T1[b1] - T1[a]) - (int64_t)a * (Cb1 - Ca) + (int64_t)cm * (Cb2 - Cb1);
      if (a > 0) nq += R - Ca;
    }
    acc += (int64_t)cm * nq;
  }
  return acc;
}

template <int D>
__device__ __forceinline__ int64_t prefix_bound(const InstSums &s, int64_t c, int64_t l,
                                                int64_t acc) {
  int64_t S;
  if (D == kMT) S = mt_sum(s, c, (uint64_t)(2 * acc));
  else if (D == kCCM1) S = ccm1_sum(s, (int64_t)((uint32_t)c / (uint32_t)l), acc);
  else S = bj1_sum(s, acc);
  const int64_t q = (D == kMT) ? 0 : (int64_t)((uint32_t)c / (uint32_t)l);
  return ceil_div_fast(S, dff_at_c_q(D, l, c, q));
}

// Builds the tables of DFF D for instance I and evaluates lambdas
// [lam0, lam_end); returns the thread's best key.
template <int MODE, int D>
__device__ unsigned long long prefix_tile_dff(const EvalArgs &A, const InstView &I, int64_t lam0,
                                              int64_t lam_end, int32_t *tab, uint32_t *s_load,
                                              PrefixShared &S) {
  const int tid = threadIdx.x;
  const int64_t c = I.c;
  const int nU = (int)prefix_u_len(c), nW = (int)prefix_w_len(c);
  int32_t *T0 = tab;
  int32_t *T1 = tab + nW;  // BJ1 only
  const int nzero = (D == kBJ1) ? 2 * nW : nU;
  for (int i = tid; i < nzero; i += kPrefixNT) tab[i] = 0;
  if (tid < 8) S.sums[tid] = 0;
  __syncthreads();

  // ---- histogram the instance's items ----------------------------------------
  int64_t ls[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t L = stream_len<MODE>(I);
  for (int64_t q = tid; q < L; q += kPrefixNT) {
    int64_t w = 0;
    if (!fetch_item<MODE>(A, I, s_load, q, w)) continue;
    if (w < 0 || w > c) {
      S.err = 1;
      continue;
    }
    ls[5] += w;
    ls[7] += 1;
    if (D == kBJ1) {
      atomicAdd(&T0[w], 1);
      atomicAdd(&T1[w], (int32_t)w);
      continue;
    }
    if (w == 0) continue;
    if (w == c) {
      ls[3]++;
    } else if (2 * w < c) {
      ls[0]++;
      atomicAdd(&T0[w], D == kMT ? (int32_t)w : 1);
    } else if (2 * w > c) {
      const int64_t u = c - w;
      ls[1]++;
      ls[4] += w;
      ls[6] += u;
      atomicAdd(&T0[u], D == kMT ? -(int32_t)u : -1);
    } else {
      ls[2]++;
    }
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const long long x = warp_sum((long long)ls[e]);
    if (lane_id() == 0 && x != 0) atomicAdd((unsigned long long *)&S.sums[e], (unsigned long long)x);
  }
  __syncthreads();
  if (D == kBJ1) {
    block_scan_i32<false>(T0, nW, S.seg);
    block_scan_i32<false>(T1, nW, S.seg);
  } else {
    block_scan_i32<true>(T0, nU, S.seg);
  }
  if (S.err) return 0ull;

  InstSums sums;
  sums.n_small = S.sums[0];
  sums.n_big = S.sums[1];
  sums.n_half = S.sums[2];
  sums.n_full = S.sums[3];
  sums.sumw_big = S.sums[4];
  sums.sumw = S.sums[5];
  const int64_t TB = S.sums[6];
  const int64_t R = S.sums[7];
  int64_t lo_d, hi_d;
  param_range(D, c, lo_d, hi_d);
  const uint32_t gbase = flat_index(D, lo_d, c);
  unsigned long long best = 0ull;

  // ---- heavy parameters (many lookups): the whole CTA shares their blocks ----
  int64_t heavy_end = lam0;
  if (D == kCCM1) heavy_end = max(lam0, min(lam_end, (prefix_u_len(c) - 2) / kHeavyBlocks + 1));
  if (D == kBJ1) heavy_end = max(lam0, min(lam_end, c / kHeavyBlocks + 1));
  heavy_end = min(heavy_end, lam0 + kMaxHeavy);
  const int nheavy = (int)(heavy_end - lam0);
  if (nheavy > 0) {
    for (int i = tid; i < nheavy; i += kPrefixNT) S.heavy_acc[i] = 0ull;
    __syncthreads();
    for (int i = 0; i < nheavy; ++i) {
      const int64_t l = lam0 + i;
      if (D == kBJ1 && (uint32_t)c % (uint32_t)l == 0) continue;  // c mod l = 0: every BJ1 term is 0
      long long part = prefix_acc<D>(T0, T1, c, l, tid, kPrefixNT, R, TB);
      part = warp_sum(part);
      if (lane_id() == 0 && part != 0)
        atomicAdd(&S.heavy_acc[i], (unsigned long long)part);
    }
    __syncthreads();
    for (int i = tid; i < nheavy; i += kPrefixNT) {
      const int64_t l = lam0 + i;
      const int64_t acc = (int64_t)S.heavy_acc[i];
      const unsigned long long key = make_key(prefix_bound<D>(sums, c, l, acc),
                                              gbase + (uint32_t)(l - lo_d));
      best = key > best ? key : best;
    }
  }
  // ---- light parameters: one thread each ----------------------------------------
  for (int64_t l = heavy_end + tid; l < lam_end; l += kPrefixNT) {
    const int64_t acc =
        (D == kBJ1 && (uint32_t)c % (uint32_t)l == 0) ? 0 : prefix_acc<D>(T0, T1, c, l, 0, 1, R, TB);
    const unsigned long long key = make_key(prefix_bound<D>(sums, c, l, acc),
                                            gbase + (uint32_t)(l - lo_d));
    best = key > best ? key : best;
  }
  return best;
}

// Persistent kernel over the prefix tile table (instance, DFF in {MT, CCM1,
// BJ1} routed here by prefix_handles, A.plpt consecutive lambdas).
template <int MODE>
__global__ void __launch_bounds__(kPrefixNT, 2) prefix_kernel(EvalArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PrefixShared S;
  __shared__ long long s_tile, s_inst;
  int32_t *tab = reinterpret_cast<int32_t *>(smem_raw);
  uint32_t *s_load = reinterpret_cast<uint32_t *>(smem_raw + kPrefixSmemBytes);

  const int64_t total = A.ptile_start ? A.ptile_start[A.B] : A.single_ptiles;
  int64_t t = blockIdx.x;
  if (A.pwork) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(A.pwork, 1ull);
    __syncthreads();
    t = s_tile;
  }
  while (t < total) {
    if (threadIdx.x == 0) {
      int64_t b = 0;
      if (A.ptile_start) {
        int64_t lo = 0, hi = A.B - 1;
        while (lo < hi) {
          const int64_t mid = (lo + hi + 1) >> 1;
          if (A.ptile_start[mid] <= t) lo = mid;
          else hi = mid - 1;
        }
        b = lo;
      }
      s_inst = b;
    }
    __syncthreads();
    const int64_t b = s_inst;
    const InstView I = resolve_instance<MODE>(A, b);
    const int64_t t0 = A.ptile_start ? A.ptile_start[b] : 0;
    const int64_t ntiles = instance_tiles(A, b);
    // which DFF and lambdas
    int64_t rem = t - t0;
    int d = 0;
    const int64_t sb = sum_bound<MODE>(I);
    for (d = 0; d < kNumDff; ++d) {
      if (!prefix_handles(d, I.c, sb, A.prefix_on)) continue;
      const int64_t nt = (param_count(d, I.c) + A.plpt - 1) / A.plpt;
      if (rem < nt) break;
      rem -= nt;
    }
    int64_t lo_d, hi_d;
    param_range(d, I.c, lo_d, hi_d);
    const int64_t lam0 = lo_d + rem * A.plpt;
    const int64_t lam_end = min(hi_d + 1, lam0 + A.plpt);

    if (threadIdx.x == 0) S.err = 0;
    __syncthreads();
    node_loads<kPrefixNT, MODE>(I, s_load, &S.err);
    __syncthreads();
    unsigned long long best;
    if (d == kMT) best = prefix_tile_dff<MODE, kMT>(A, I, lam0, lam_end, tab, s_load, S);
    else if (d == kCCM1) best = prefix_tile_dff<MODE, kCCM1>(A, I, lam0, lam_end, tab, s_load, S);
    else best = prefix_tile_dff<MODE, kBJ1>(A, I, lam0, lam_end, tab, s_load, S);
    __syncthreads();
    fold_and_finalize<kPrefixNT>(A, b, best, S.err != 0, ntiles, I, S.warp_key);
    if (!A.pwork) break;
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(A.pwork, 1ull);
    __syncthreads();
    t = s_tile;
  }
}

}  // namespace bplb
