// bp_lb_prefix.cuh -- prefix-count evaluation of MT, RAD2, CCM1 and BJ1.
//
// Same bounds as the direct evaluators (bit-exact), asymptotically less work:
// per tile the instance's items are histogrammed by value in shared memory and
// suffix-scanned, after which each parameter needs O(1) (MT, RAD2), O(U / l)
// (CCM1) or O(c / l) (BJ1) table lookups instead of one evaluation per item.
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
//         it is sum_j (NN(j l + 1) - NN(j l + cm + 1)) over j = 0 .. floor(c / l).
// NN is the suffix sum of the suffix count N(x) = #[w >= x]: a histogram
// scanned twice.  Every table entry and every sum above is bounded by the
// instance's size total, below 2^31 on this path (prefix_handles), so the
// tables and accumulators are 32-bit.  VB2 and FS1 stay on the direct kernel.
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
constexpr uint32_t kCtaBlocks = kPrefixNT;
constexpr uint32_t kWarpBlocks = 32;
constexpr int kMaxHeavy = kPrefixNT;

struct PrefixShared {
  int err;
  int pad_;
  unsigned long long warp_key[kPrefixWarps];
  long long sums[8];  // n_small, n_big, n_half, n_full, sumw_big, sumw, total big u, unused
  uint32_t wtot[2][kPrefixWarps];
  uint32_t heavy_acc[kMaxHeavy];
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
template <bool TWICE>
__device__ void suffix_scan(int32_t *a, int n, PrefixShared &S) {
  const int per = ((n + kPrefixNT - 1) / kPrefixNT) | 1;
  const int s0 = min(n, (int)threadIdx.x * per), s1 = min(n, s0 + per);
  uint32_t h = 0, m = 0;
  for (int i = s0; i < s1; ++i) {
    const uint32_t v = (uint32_t)a[i];
    h += v;
    if (TWICE) m += v * (uint32_t)(i - s0 + 1);  // this segment's part of the twice-scanned a[s0]
  }
  const uint32_t n_after = block_sum_after(h, S.wtot[0]);
  uint32_t nn_after = 0;
  if (TWICE) nn_after = block_sum_after(m + (uint32_t)(s1 - s0) * n_after, S.wtot[1]);
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

// Table geometry and constants of one tile.
struct PrefixCtx {
  InstSums s;
  int64_t c;
  int64_t TB;     // sum of u over big items
  uint32_t U;     // floor((c - 1) / 2): largest small or big u
  uint32_t U1;    // U + 1: the zero sentinel of the u-domain tables
  int64_t lo_d;   // first parameter of the DFF
  uint32_t gbase; // its flattened index
};

// Lookup blocks of one parameter (D = CCM1 or BJ1): b0, b0 + bs, ...
//   CCM1: block b is x = (b + 1) l <= U, term N'(x);
//   BJ1:  block b is x = b l + 1 <= c, term NN(x) - NN(x + cm)  (cm > 0).
template <int D>
__device__ __forceinline__ uint32_t block_terms(const int32_t *T, uint32_t c32, uint32_t U,
                                                uint32_t l, uint32_t cm, uint32_t b0, uint32_t bs) {
  const uint32_t step = bs * l;
  uint32_t acc = 0;
  if (D == kCCM1) {
    uint32_t x = (b0 + 1u) * l;
#pragma unroll 4
    for (; x <= U; x += step) acc += (uint32_t)T[x];
  } else {
    uint32_t x = b0 * l + 1u;
#pragma unroll 4
    for (; x <= c32; x += step) acc += (uint32_t)(T[x] - T[x + cm]);
  }
  return acc;
}

// Sum S(l) and denominator f(c, l) from the accumulator, and the candidate
// test against the thread's best bound B (see the file comment).
template <int D>
__device__ __forceinline__ void consider(const PrefixCtx &x, uint32_t l, int64_t acc, int64_t &B,
                                         unsigned long long &best) {
  const int64_t c = x.c;
  int64_t S, f;
  if (D == kMT) {
    S = mt_sum(x.s, c, (uint64_t)(2 * acc));
    f = c;
  } else if (D == kRAD2) {
    S = acc;  // assembled by the caller
    f = c;
  } else {
    const uint32_t q = (uint32_t)c / l;
    if (D == kCCM1) {
      S = ccm1_sum(x.s, (int64_t)q, acc);
      f = 2 * (int64_t)q;
    } else {
      S = bj1_sum(x.s, acc);
      f = (int64_t)q * (int64_t)(l - ((uint32_t)c - q * l));
    }
  }
  if (S > B * f || (D == kMT && l == 0u)) {
    const int64_t lb = ceil_div_fast(S, f);
    B = lb;
    best = make_key(lb, x.gbase + (uint32_t)((int64_t)l - x.lo_d));
  }
}

// Builds the table(s) of DFF D for instance I and evaluates parameters
// [lam0, lam_end); returns the thread's best key.
template <int MODE, int D>
__device__ unsigned long long prefix_tile_dff(const EvalArgs &A, const InstView &I, int64_t lam0,
                                              int64_t lam_end, int32_t *tab, uint32_t *s_load,
                                              PrefixShared &S) {
  const int tid = threadIdx.x;
  const int64_t c = I.c;
  const uint32_t c32 = (uint32_t)c;
  const uint32_t U = (uint32_t)((c - 1) / 2);
  const int nU = (int)U + 2, nW = (int)c + 2;
  int32_t *T0 = tab;       // E, N', N' or NN
  int32_t *T1 = tab + nU;  // RAD2: Ns
  const int nzero = (D == kBJ1) ? nW : (D == kRAD2 ? 2 * nU : nU);
  {
    int4 *t4 = reinterpret_cast<int4 *>(tab);
    const int4 z = make_int4(0, 0, 0, 0);
    for (int i = tid; i < (nzero + 3) / 4; i += kPrefixNT) t4[i] = z;
  }
  if (tid < 8) S.sums[tid] = 0;
  __syncthreads();

  // ---- histogram the instance's items ----------------------------------------
  int64_t ls[7] = {0, 0, 0, 0, 0, 0, 0};
  const int64_t L = stream_len<MODE>(I);
  for (int64_t q = tid; q < L; q += kPrefixNT) {
    int64_t w = 0;
    if (!fetch_item<MODE>(A, I, s_load, q, w)) continue;
    if (w < 0 || w > c) {
      S.err = 1;
      continue;
    }
    ls[5] += w;
    if (D == kBJ1) {
      atomicAdd(&T0[w], 1);
      continue;
    }
    if (w == 0) continue;
    if (w == c) {
      ls[3]++;
    } else if (2 * w < c) {
      ls[0]++;
      atomicAdd(&T0[w], D == kMT ? (int32_t)w : 1);
      if (D == kRAD2) atomicAdd(&T1[w], 1);
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
  for (int e = 0; e < 7; ++e) {
    const long long x = warp_sum((long long)ls[e]);
    if (lane_id() == 0 && x != 0) atomicAdd((unsigned long long *)&S.sums[e], (unsigned long long)x);
  }
  __syncthreads();
  if (D == kBJ1) {
    suffix_scan<true>(T0, nW, S);
  } else {
    suffix_scan<false>(T0, nU, S);
    if (D == kRAD2) suffix_scan<false>(T1, nU, S);
  }
  if (S.err) return 0ull;

  PrefixCtx x;
  x.s.n_small = S.sums[0];
  x.s.n_big = S.sums[1];
  x.s.n_half = S.sums[2];
  x.s.n_full = S.sums[3];
  x.s.sumw_big = S.sums[4];
  x.s.sumw = S.sums[5];
  x.TB = S.sums[6];
  x.c = c;
  x.U = U;
  x.U1 = U + 1u;
  int64_t hi_d;
  param_range(D, c, x.lo_d, hi_d);
  x.gbase = flat_index(D, x.lo_d, c);
  int64_t B = ceil_div_fast(x.s.sumw, c);  // L1
  unsigned long long best = 0ull;

  if (D == kMT || D == kRAD2) {
    for (int64_t l = lam0 + tid; l < lam_end; l += kPrefixNT) {
      const uint32_t l32 = (uint32_t)l;
      int64_t acc;
      if (D == kMT) {
        acc = (int64_t)T0[min(l32, x.U1)] + x.TB;
      } else {
        const uint32_t y = min(c32 - 2u * l32 + 1u, x.U1);
        const int64_t n1 = T0[l32], n2s = T1[y], n2b = (int64_t)T1[y] - T0[y];
        acc = rad2_sum(x.s, c, n1, n2s, n2b);
      }
      consider<D>(x, l32, acc, B, best);
    }
    return best;
  }

  // CCM1 / BJ1: lookups per parameter fall like X / l.
  const uint32_t X = (D == kCCM1) ? U : c32;
  const int64_t cta_end = max(lam0, min(lam_end, min((int64_t)(X / kCtaBlocks) + 1, lam0 + kMaxHeavy)));
  const int64_t warp_end = max(cta_end, min(lam_end, (int64_t)(X / kWarpBlocks) + 1));
  const int lane = (int)lane_id(), warp = tid >> 5;

  // ---- parameters shared by the whole CTA ---------------------------------------
  const int ncta = (int)(cta_end - lam0);
  if (ncta > 0) {
    for (int i = tid; i < ncta; i += kPrefixNT) S.heavy_acc[i] = 0u;
    __syncthreads();
    for (int i = 0; i < ncta; ++i) {
      const uint32_t l = (uint32_t)(lam0 + i);
      const uint32_t cm = c32 % l;
      if (D == kBJ1 && cm == 0u) continue;  // every BJ1 term is 0
      const uint32_t part = warp_sum(block_terms<D>(T0, c32, U, l, cm, (uint32_t)tid, kPrefixNT));
      if (lane == 0 && part != 0u) atomicAdd(&S.heavy_acc[i], part);
    }
    __syncthreads();
    if (tid < ncta) {
      const uint32_t l = (uint32_t)(lam0 + tid);
      const int64_t acc = (D == kCCM1) ? (int64_t)(int32_t)S.heavy_acc[tid] : (int64_t)S.heavy_acc[tid];
      consider<D>(x, l, acc, B, best);
    }
  }

  // ---- parameters shared by one warp (lane t of a round of 32 keeps the t-th) ---
  {
    const int64_t nwarp = warp_end - cta_end;
    // warp w takes the parameters cta_end + w + 8 i, i = 0, 1, ...
    const int64_t mine_n = nwarp > warp ? (nwarp - warp + kPrefixWarps - 1) / kPrefixWarps : 0;
    for (int64_t r0 = 0; r0 < mine_n; r0 += 32) {
      uint32_t mine = 0;
      const int cnt = (int)min((int64_t)32, mine_n - r0);
      for (int t = 0; t < cnt; ++t) {
        const uint32_t l = (uint32_t)(cta_end + warp + (r0 + t) * kPrefixWarps);
        const uint32_t cm = c32 % l;
        uint32_t part = 0;
        if (D == kCCM1 || cm != 0u) part = warp_sum(block_terms<D>(T0, c32, U, l, cm, (uint32_t)lane, 32u));
        if (lane == t) mine = part;
      }
      if (lane < cnt) {
        const uint32_t l = (uint32_t)(cta_end + warp + (r0 + lane) * kPrefixWarps);
        consider<D>(x, l, D == kCCM1 ? (int64_t)(int32_t)mine : (int64_t)mine, B, best);
      }
    }
  }

  // ---- one thread per parameter; alternate directions balance the rounds --------
  for (int64_t r = warp_end; r < lam_end; r += kPrefixNT) {
    const int64_t round = (r - warp_end) / kPrefixNT;
    const int64_t l = r + ((round & 1) ? kPrefixNT - 1 - tid : tid);
    if (l >= lam_end) continue;
    const uint32_t l32 = (uint32_t)l;
    const uint32_t cm = c32 % l32;
    uint32_t acc = 0;
    if (D == kCCM1 || cm != 0u) acc = block_terms<D>(T0, c32, U, l32, cm, 0u, 1u);
    consider<D>(x, l32, D == kCCM1 ? (int64_t)(int32_t)acc : (int64_t)acc, B, best);
  }
  return best;
}

// Persistent kernel over the prefix tile table (instance, DFF in {MT, RAD2,
// CCM1, BJ1} routed here by prefix_handles, A.plpt consecutive lambdas).
template <int MODE>
__global__ void __launch_bounds__(kPrefixNT, 4) prefix_kernel(EvalArgs A) {
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
    else if (d == kRAD2) best = prefix_tile_dff<MODE, kRAD2>(A, I, lam0, lam_end, tab, s_load, S);
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
