// bp_lb_l2.cuh -- Martello and Toth's L2 (Sec. 3.1) on the device, the
// comparator of the DFF bounds.
//
// L2(I, l) = |W1| + |W2| + max(0, ceil((sum W3 - (c |W2| - sum W2)) / c)) with
// W1 = {w > c - l}, W2 = {c/2 < w <= c - l}, W3 = {l <= w <= c/2}, maximised
// over integer l in [0, floor(c/2)] (the integer reading of the parameter).
// The three sets, hence L2(I, l), change only where l passes an item: W3
// loses w at l = w + 1 and W1 gains w at l = c - w + 1.  So the maximum is
// taken over l = 0 and those breakpoints (at most 2r + 1 values, each the
// start of an interval on which L2(I, l) is constant).  Per instance one CTA
// sorts the items in shared memory (bitonic), forms their prefix sums, and
// evaluates every breakpoint with two binary searches: O(r log r) work.
#pragma once

#include "bp_lb_kernels.cuh"

namespace bplb {

constexpr int kL2NT = 256;
constexpr int kL2MaxItems = 8192;
constexpr size_t kL2SmemBytes = sizeof(uint32_t) * kL2MaxItems + sizeof(int64_t) * (kL2MaxItems + 1);

// First index in v[0..n) (ascending) with v[i] > x, for x in [-1, 2^32 - 2].
__device__ __forceinline__ int upper_index(const uint32_t *v, int n, int64_t x) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)v[mid] > x) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <int NT>
__global__ void __launch_bounds__(NT) l2_kernel(int32_t B, const int64_t *offsets,
                                                const int32_t *sizes, const int64_t *capacity,
                                                int64_t *out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *key = reinterpret_cast<uint32_t *>(smem_raw);
  int64_t *pre = reinterpret_cast<int64_t *>(smem_raw + sizeof(uint32_t) * kL2MaxItems);
  __shared__ int s_err;
  __shared__ unsigned long long s_best;
  __shared__ int64_t s_tot[NT / 32];
  const int tid = threadIdx.x;

  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    const int64_t c = capacity[b];
    const int64_t beg = offsets[b];
    const int64_t r64 = offsets[b + 1] - beg;
    if (c < 1 || c > kMaxCapacity || r64 < 0 || r64 > kL2MaxItems) {  // same for every thread
      if (tid == 0) out[b] = -BP_ERANGE;
      continue;
    }
    const int r = (int)r64;
    int P = 1;
    while (P < r) P <<= 1;
    if (tid == 0) {
      s_err = 0;
      s_best = 0ull;
    }
    __syncthreads();
    for (int i = tid; i < P; i += NT) {
      uint32_t v = 0xFFFFFFFFu;  // padding sorts to the end
      if (i < r) {
        const int32_t w = sizes[beg + i];
        if (w < 0 || (int64_t)w > c) s_err = 1;
        v = (uint32_t)max(w, 0);
      }
      key[i] = v;
    }
    __syncthreads();
    // ---- bitonic sort, ascending -------------------------------------------------
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < P; i += NT) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const uint32_t a = key[i], d = key[ixj];
            if ((a > d) == ((i & k) == 0)) {
              key[i] = d;
              key[ixj] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    // ---- exclusive prefix sums pre[0..r] of the sorted items -------------------------
    {
      const int per = (r + NT - 1) / NT;
      const int s0 = min(r, tid * per), s1 = min(r, s0 + per);
      int64_t tot = 0;
      for (int i = s0; i < s1; ++i) tot += key[i];
      int64_t x = tot;  // inclusive scan of the segment totals within the warp
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if ((int)lane_id() >= o) x += y;
      }
      if (lane_id() == 31) s_tot[tid >> 5] = x;
      __syncthreads();
      int64_t run = x - tot;
      for (int w = 0; w < (tid >> 5); ++w) run += s_tot[w];
      for (int i = s0; i < s1; ++i) {
        pre[i] = run;
        run += key[i];
      }
      if (s1 == r && s0 < s1) pre[r] = run;  // the thread whose segment ends the list
      if (r == 0 && tid == 0) pre[0] = 0;
    }
    __syncthreads();
    if (!s_err) {
      const int64_t H = c / 2;
      const int m = upper_index(key, r, H);  // items with w <= c/2 come first
      const int64_t pre_m = pre[m];
      unsigned long long best = 0ull;
      for (int i = tid; i < 2 * r + 1; i += NT) {
        int64_t l;
        if (i == 2 * r) l = 0;
        else if (i < r) l = (int64_t)key[i] + 1;        // W3 loses key[i] here
        else l = c - (int64_t)key[i - r] + 1;            // W1 gains key[i - r] here
        if (l < 0 || l > H) continue;
        const int ub = upper_index(key, r, c - l);       // items > c - l: W1
        const int64_t n1 = r - ub, n2 = ub - m;          // W2: c/2 < w <= c - l
        const int64_t s2 = pre[ub] - pre_m;
        const int lo = upper_index(key, r, l - 1);       // first item >= l
        const int64_t s3 = pre_m - pre[lo];              // W3: l <= w <= c/2
        const int64_t num = s3 - (c * n2 - s2);
        const int64_t v = n1 + n2 + (num > 0 ? (num + c - 1) / c : 0);
        best = max(best, (unsigned long long)v);
      }
      best = warp_max_u64(best);
      if (lane_id() == 0) atomicMax(&s_best, best);
    }
    __syncthreads();
    if (tid == 0) out[b] = s_err ? -BP_ERANGE : (int64_t)s_best;
    __syncthreads();
  }
}

}  // namespace bplb
