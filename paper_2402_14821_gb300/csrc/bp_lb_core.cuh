// bp_lb_core.cuh -- device building blocks of the DFF lower-bound check.
//
// Method: Tardivo, Michel, Pontelli, arXiv 2402.14821, Sec. 3.1 (the six
// dual-feasible functions), Alg. 2 (the collection of L1-like bounds) and
// Alg. 4 (one parameter per GPU thread, items held in shared memory).
//
// Everything here is exact integer arithmetic.  The per-item work is written
// as exact rearrangements of the printed case analyses (each one derived in
// the comment above its evaluator), so that the inner loops need no data-
// dependent branches:
//
//   Items are classified once per instance (independently of lambda):
//     w == 0       contributes f(0, lambda) = 0 to every DFF: dropped;
//     w == c       contributes exactly f(c, lambda): counted (n_full);
//     2w <  c      "small", stored as u2 = 2w        (u = w);
//     2w >  c      "big",   stored as u2 = 2(c - w)  (u = c - w);
//     2w == c      "half":  counted (n_half).
//   MT, RAD2, CCM1 and VB2 depend on w only through u and its class; FS1 and
//   BJ1 use the raw sizes (stored as w or 2w).  Sizes are kept doubled where
//   the exact division below needs an even numerator.
//
//   Exact division by an invariant divisor d < 2^31 of a numerator n < 2^31
//   (Granlund & Montgomery, "Division by invariant integers using
//   multiplication", PLDI 1994, Thm. 4.2 with N = 31):
//     l = ceil(log2 d), m = ceil(2^(31+l) / d)  (m < 2^32),
//     floor(n / d) = floor(m * n / 2^(31+l)) = umulhi(2n, m) >> l.
#pragma once

#include <cstdint>

#define BPLB_HD __host__ __device__ __forceinline__
#define BPLB_D __device__ __forceinline__

namespace bplb {

constexpr int kNumDff = 6;
enum : int { kMT = 0, kRAD2 = 1, kFS1 = 2, kCCM1 = 3, kVB2 = 4, kBJ1 = 5 };

constexpr int64_t kMaxCapacity = int64_t(1) << 30;
constexpr int64_t kMaxItems = int64_t(1) << 20;
// Fast-path limits (the generic 64-bit path takes over above them).
constexpr int64_t kNarrowCap = int64_t(1) << 28;   // 32-bit partial sums, all DFFs
constexpr int64_t kVb2FixedCap = 65535;            // (l + 1) c < 2^32 for l <= c
constexpr int64_t kVb2FloatCap = int64_t(1) << 22; // fp32 quotient estimate exact
constexpr int64_t kFs1FastCap = 21262214;          // 101 * c < 2^31
constexpr int64_t kCcm1NoShiftCap = 131071;        // u e < (c/2)^2 < 2^32
constexpr int64_t kBj1NoShiftCap = 65535;          // w e < c^2 < 2^32

// ---------------------------------------------------------------------------
// Parameter ranges (Sec. 3.1, integer lambda):
//   MT [0, c/2]; RAD2 (c/4, c/3]; FS1 [1, 100]; CCM1 [1, c/2]; VB2 [2, c];
//   BJ1 [1, c].
// ---------------------------------------------------------------------------
BPLB_HD void param_range(int d, int64_t c, int64_t &lo, int64_t &hi) {
  switch (d) {
    case kMT:   lo = 0;         hi = c / 2; break;
    case kRAD2: lo = c / 4 + 1; hi = c / 3; break;
    case kFS1:  lo = 1;         hi = 100;   break;
    case kCCM1: lo = 1;         hi = c / 2; break;
    case kVB2:  lo = 2;         hi = c;     break;
    default:    lo = 1;         hi = c;     break;  // kBJ1
  }
}

BPLB_HD int64_t param_count(int d, int64_t c) {
  int64_t lo, hi;
  param_range(d, c, lo, hi);
  return hi >= lo ? hi - lo + 1 : 0;
}

BPLB_HD int64_t param_total(int64_t c) {
  int64_t t = 0;
  for (int d = 0; d < kNumDff; ++d) t += param_count(d, c);
  return t;
}

// Tiles of `lpt` parameters per DFF, DFFs in paper order.
BPLB_HD int64_t tiles_for(int64_t c, int64_t lpt) {
  int64_t t = 0;
  for (int d = 0; d < kNumDff; ++d) t += (param_count(d, c) + lpt - 1) / lpt;
  return t;
}

// ---------------------------------------------------------------------------
// Exact division by an invariant 31-bit divisor (see file comment).
// ---------------------------------------------------------------------------
struct Div31 {
  uint32_t m;
  uint32_t l;
};

BPLB_HD uint32_t ceil_log2_u32(uint32_t d) {
#ifdef __CUDA_ARCH__
  return d <= 1 ? 0u : 32u - (uint32_t)__clz(d - 1);
#else
  uint32_t l = 0;
  while (l < 32 && (uint64_t(1) << l) < d) ++l;
  return l;
#endif
}

BPLB_HD Div31 div31_make(uint32_t d) {
  Div31 r;
  r.l = ceil_log2_u32(d);
  const uint64_t num = uint64_t(1) << (31 + r.l);
  r.m = (uint32_t)((num + d - 1) / d);
  return r;
}

// Division without the final shift, for small numerators: with
// m1 = ceil(2^32 / d) (d >= 2) and e = m1 d - 2^32 < d,
//   n m1 / 2^32 = n / d + n e / (d 2^32),
// so floor(n m1 / 2^32) = floor(n / d) whenever n e < 2^32, in particular
// whenever n d < 2^32.  For d = 1 the magic 2^32 does not fit; m1 = 2^32 - 1
// then gives n - 1 for n >= 1 (and 0 for n = 0), which callers correct.
// ceil(2^32 / d) = floor((2^32 - 1) / d) + 1 for d >= 2 (one 32-bit division).
BPLB_HD uint32_t div_noshift_make(uint32_t d) {
  return d <= 1 ? 0xFFFFFFFFu : 0xFFFFFFFFu / d + 1u;
}

// floor(n / d) given n2 = 2n (n < 2^31).
BPLB_HD uint32_t div31(uint32_t n2, Div31 D) {
#ifdef __CUDA_ARCH__
  return __umulhi(n2, D.m) >> D.l;
#else
  return (uint32_t)(((uint64_t)n2 * D.m) >> 32) >> D.l;
#endif
}

// ---------------------------------------------------------------------------
// Per-instance constants gathered while staging (all lambda-independent).
// ---------------------------------------------------------------------------
struct InstSums {
  int64_t n_small;   // items with 0 < 2w < c
  int64_t n_big;     // items with c < 2w < 2c
  int64_t n_half;    // items with 2w == c
  int64_t n_full;    // items with w == c
  int64_t sumw_big;  // sum of w over big items
  int64_t sumw;      // sum of w over all items
};

BPLB_HD int64_t ceil_div_i64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ceil(a / b) for 0 <= a, 0 < b, with a 32-bit division whenever both fit.
BPLB_HD int64_t ceil_div_fast(int64_t a, int64_t b) {
  if (((uint64_t)a >> 32) == 0 && ((uint64_t)b >> 32) == 0) {
    const uint32_t q = (uint32_t)a / (uint32_t)b;
    return (int64_t)q + ((uint32_t)a != q * (uint32_t)b);
  }
  return (a + b - 1) / b;
}

// ---------------------------------------------------------------------------
// S(d, lambda) = sum_i f_d(w_i, lambda) assembled from one lambda-dependent
// list accumulator (defined next to each evaluator in bp_lb_eval.cuh) and the
// lambda-independent instance sums.  Each identity below is an exact
// rearrangement of the printed case analysis (Sec. 3.1).
// ---------------------------------------------------------------------------

// f_MT(w, l) = c if w > c - l; w if l <= w <= c - l; 0 if w < l (l <= c/2).
//   small (w = u < c/2 <= c - l):  u * [u >= l]
//   big   (w > c/2 >= l):          w + u * [u < l]   (u = c - w; w > c - l <=> u < l)
//   half  (w = c/2):               c/2
//   full:                          c = f(c)
// acc = sum_small u2*[u2 >= 2l] + sum_big u2*[u2 < 2l]   (u2 = 2u).
BPLB_HD int64_t mt_sum(const InstSums &s, int64_t c, uint64_t acc) {
  return (int64_t)(acc >> 1) + s.sumw_big + s.n_half * (c / 2) + s.n_full * c;
}

// f_RAD2, c/4 < l <= c/3, A = floor(c/3), B = floor(c/2):
//   small: 0 (u < l), A (l <= u <= c-2l), B (c-2l < u; always < 2l)
//        = A*[u >= l] + (B - A)*[u > c - 2l]           (c - 2l >= l)
//   big:   w < 2l <=> u > c - 2l: B;  else c - f(u): c - A (u >= l) or c (u < l)
//        = c - A*[u >= l] - (c - A - B)*[u > c - 2l]
//   half:  B;  full: c.
// n1 = #small[u >= l] - #big[u >= l]; n2s, n2b = #[u > c - 2l] per list.
BPLB_HD int64_t rad2_sum(const InstSums &s, int64_t c, int64_t n1, int64_t n2s, int64_t n2b) {
  const int64_t A = c / 3, B = c / 2;
  return A * n1 + (B - A) * n2s + s.n_big * c - (c - A - B) * n2b + s.n_half * B + s.n_full * c;
}

// f_FS1(w, l) = w*l if c | w(l+1), else c*floor(w(l+1)/c)
//            = c*floor(w(l+1)/c) - w*[c | w(l+1)]   (raw sizes, all items).
// acc = sum of that expression.
BPLB_HD int64_t fs1_sum(int64_t acc) { return acc; }

// f_CCM1, Q = floor(c/l): big 2Q - 2 floor(u/l); half Q; small 2 floor(u/l); full 2Q.
// acc = sum_small floor(u/l) - sum_big floor(u/l).
BPLB_HD int64_t ccm1_sum(const InstSums &s, int64_t Q, int64_t acc) {
  return 2 * acc + Q * (2 * s.n_big + s.n_half + 2 * s.n_full);
}

// f_VB2 with ceil(c*l/c) = l and g(u) = max(0, ceil(u*l/c) - 1) = ceil(u*l/c) - 1 for u >= 1:
//   small 2 g(u); big 2(l-1) - 2 g(u); half l - 1; full 2(l-1) = f(c).
// acc = sum_small ceil(u*l/c) - sum_big ceil(u*l/c)  (every listed u >= 1).
BPLB_HD int64_t vb2_sum(const InstSums &s, int64_t l, int64_t acc) {
  return 2 * (acc - s.n_small + s.n_big) + (l - 1) * (2 * s.n_big + s.n_half + 2 * s.n_full);
}

// f_BJ1 with q = floor(w/l), rho = w mod l, cm = c mod l:
//   q(l - cm) + max(0, rho - cm) = w - (cm*q + min(rho, cm))    (w = q l + rho).
// acc = sum (cm*q + min(rho, cm))  (raw sizes, all items).
BPLB_HD int64_t bj1_sum(const InstSums &s, int64_t acc) { return s.sumw - acc; }

// f(c, lambda) of each DFF (Sec. 3.1): the denominator of the bound.  > 0 on
// every parameter range: MT c, RAD2 c, FS1 c*l, CCM1 2 floor(c/l) >= 4,
// VB2 2(l - 1) >= 2, BJ1 floor(c/l)(l - c mod l) >= 1.
BPLB_HD int64_t dff_at_c(int d, int64_t l, int64_t c) {
  switch (d) {
    case kMT:
    case kRAD2: return c;
    case kFS1:  return c * l;
    case kCCM1: return 2 * (c / l);
    case kVB2:  return 2 * (l - 1);
    default:    return (c / l) * (l - c % l);
  }
}

// The same with c / l given (both < 2^31, so the caller divides in 32 bits).
BPLB_HD int64_t dff_at_c_q(int d, int64_t l, int64_t c, int64_t q) {
  switch (d) {
    case kMT:
    case kRAD2: return c;
    case kFS1:  return c * l;
    case kCCM1: return 2 * q;
    case kVB2:  return 2 * (l - 1);
    default:    return q * (l - (c - q * l));
  }
}

// Flattened parameter index g (paper order, lambda ascending) and its inverse.
BPLB_HD uint32_t flat_index(int d, int64_t l, int64_t c) {
  int64_t g = 0;
  for (int e = 0; e < d; ++e) g += param_count(e, c);
  int64_t lo, hi;
  param_range(d, c, lo, hi);
  return (uint32_t)(g + (l - lo));
}

BPLB_HD void unflatten(uint32_t g, int64_t c, int32_t &d, int64_t &l) {
  int64_t rem = g;
  for (int e = 0; e < kNumDff; ++e) {
    const int64_t n = param_count(e, c);
    if (rem < n) {
      int64_t lo, hi;
      param_range(e, c, lo, hi);
      d = e;
      l = lo + rem;
      return;
    }
    rem -= n;
  }
  d = 0;
  l = 0;
}

// Key whose maximum is (largest bound, then smallest flattened index).
BPLB_HD unsigned long long make_key(int64_t lb, uint32_t g) {
  return ((unsigned long long)lb << 32) | (unsigned long long)(0xFFFFFFFFu - g);
}

}  // namespace bplb
