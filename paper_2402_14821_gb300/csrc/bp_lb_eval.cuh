// bp_lb_eval.cuh -- per-DFF inner loops over one staged item list, for T
// parameters per thread (Alg. 4 gives each GPU thread one parameter; here a
// thread carries T of them so that every item read from shared memory feeds T
// independent evaluations).
//
// Lists live in shared memory as uint32 values, padded with zeros to a
// multiple of 4 so that each step reads four items with one 16-byte broadcast
// load (all lanes of a warp read the same address).  A zero pad contributes 0
// to every list sum below.
//
// Partial sums are 32-bit within a group of K items, K chosen so that the
// group's true sum stays below 2^32, then folded into one 64-bit accumulator
// per parameter with the sign (+1 small list, -1 big list) or weight the DFF's
// sum needs.  The *_wide variants accumulate in 64 bits directly; they serve
// capacities above the fast-path limits.
#pragma once

#include "bp_lb_core.cuh"

namespace bplb {

// Largest multiple of 4 not above floor((2^32 - 1) / max_term), capped at 2^30.
// Callers guarantee max_term <= 2^30 - 1 so that the result is >= 4.
BPLB_HD int group_len(int64_t max_term) {
  if (max_term < 1) max_term = 1;
  int64_t k = (int64_t)0xFFFFFFFFu / max_term;
  if (k > (int64_t(1) << 30)) k = int64_t(1) << 30;
  k &= ~int64_t(3);
  return k < 4 ? 4 : (int)k;
}

BPLB_D uint4 lds4(const uint32_t *s, int i) { return *reinterpret_cast<const uint4 *>(s + i); }
BPLB_D float4 lds4f(const float *s, int i) { return *reinterpret_cast<const float4 *>(s + i); }

// Conditional accumulate on the FMA pipe: if (pred) a += x, issued as a
// predicated integer multiply-add x * one + a.  `one` is 1 at run time (a
// kernel argument), so the compiler keeps the multiply-add instead of turning
// it into an ALU-pipe add; the compare itself stays on the ALU pipe.  Used to
// balance the two integer pipes of an SM sub-partition.
BPLB_D uint32_t add_if_ge(uint32_t a, uint32_t x, uint32_t t, uint32_t one) {
  asm("{\n\t.reg .pred p;\n\tsetp.ge.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %1, %3, %0;\n\t}"
      : "+r"(a) : "r"(x), "r"(t), "r"(one));
  return a;
}
BPLB_D uint32_t add_if_lt(uint32_t a, uint32_t x, uint32_t t, uint32_t one) {
  asm("{\n\t.reg .pred p;\n\tsetp.lt.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %1, %3, %0;\n\t}"
      : "+r"(a) : "r"(x), "r"(t), "r"(one));
  return a;
}
// if (x >= t) n += 1 / if (x > t) n += 1, as predicated multiply-adds.
BPLB_D uint32_t count_if_ge(uint32_t n, uint32_t x, uint32_t t, uint32_t one) {
  asm("{\n\t.reg .pred p;\n\tsetp.ge.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %3, %0;\n\t}"
      : "+r"(n) : "r"(x), "r"(t), "r"(one));
  return n;
}
BPLB_D uint32_t count_if_gt(uint32_t n, uint32_t x, uint32_t t, uint32_t one) {
  asm("{\n\t.reg .pred p;\n\tsetp.gt.u32 p, %1, %2;\n\t@p mad.lo.u32 %0, %3, %3, %0;\n\t}"
      : "+r"(n) : "r"(x), "r"(t), "r"(one));
  return n;
}

// ---- MT: acc += sum_small u2*[u2 >= 2l]  (BIG: sum_big u2*[u2 < 2l]) ---------
template <int T, bool BIG>
BPLB_D void mt_list(const uint32_t *s, int beg, int end, int K, const uint32_t (&thr)[T],
                    uint32_t one, uint64_t (&acc)[T]) {
  for (int g0 = beg; g0 < end; g0 += K) {
    const int g1 = min(end, g0 + K);
    uint32_t a[T];
#pragma unroll
    for (int j = 0; j < T; ++j) a[j] = 0;
#pragma unroll 2
    for (int i = g0; i < g1; i += 4) {
      const uint4 v = lds4(s, i);
#pragma unroll
      for (int j = 0; j < T; ++j) {
        if (!BIG) {
          a[j] = add_if_ge(a[j], v.x, thr[j], one);
          a[j] = add_if_ge(a[j], v.y, thr[j], one);
          a[j] = add_if_ge(a[j], v.z, thr[j], one);
          a[j] = add_if_ge(a[j], v.w, thr[j], one);
        } else {
          a[j] = add_if_lt(a[j], v.x, thr[j], one);
          a[j] = add_if_lt(a[j], v.y, thr[j], one);
          a[j] = add_if_lt(a[j], v.z, thr[j], one);
          a[j] = add_if_lt(a[j], v.w, thr[j], one);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) acc[j] += a[j];
  }
}

// ---- RAD2: n1 += #[u2 >= 2l] (SIGN), n2 += #[u2 > 2c - 4l] ---------------------
template <int T, int SIGN>
BPLB_D void rad2_list(const uint32_t *s, int beg, int end, const uint32_t (&t1)[T],
                      const uint32_t (&t2)[T], uint32_t one, int32_t (&n1)[T],
                      uint32_t (&n2)[T]) {
  uint32_t c1[T];
#pragma unroll
  for (int j = 0; j < T; ++j) c1[j] = 0;
#pragma unroll 2
  for (int i = beg; i < end; i += 4) {
    const uint4 v = lds4(s, i);
#pragma unroll
    for (int j = 0; j < T; ++j) {
      c1[j] = count_if_ge(c1[j], v.x, t1[j], one);
      c1[j] = count_if_ge(c1[j], v.y, t1[j], one);
      c1[j] = count_if_ge(c1[j], v.z, t1[j], one);
      c1[j] = count_if_ge(c1[j], v.w, t1[j], one);
      n2[j] = count_if_gt(n2[j], v.x, t2[j], one);
      n2[j] = count_if_gt(n2[j], v.y, t2[j], one);
      n2[j] = count_if_gt(n2[j], v.z, t2[j], one);
      n2[j] = count_if_gt(n2[j], v.w, t2[j], one);
    }
  }
#pragma unroll
  for (int j = 0; j < T; ++j) n1[j] += SIGN * (int32_t)c1[j];
}

// ---- FS1 (raw w): acc += c * floor(w(l+1)/c) - w*[c | w(l+1)] ----------------
template <int T>
BPLB_D void fs1_list(const uint32_t *s, int beg, int end, int K, const uint32_t (&mul2)[T],
                     Div31 Dc, uint32_t c2, int64_t c, int64_t (&acc)[T]) {
  for (int g0 = beg; g0 < end; g0 += K) {
    const int g1 = min(end, g0 + K);
    uint32_t a0[T], a1[T];
#pragma unroll
    for (int j = 0; j < T; ++j) a0[j] = a1[j] = 0;
#pragma unroll 2
    for (int i = g0; i < g1; i += 4) {
      const uint4 v = lds4(s, i);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
          const uint32_t x2 = w4[e] * mul2[j];  // 2 w (l + 1) < 2^32
          const uint32_t q = div31(x2, Dc);     // floor(w (l + 1) / c)
          a0[j] += q;
          a1[j] += (q * c2 == x2) ? w4[e] : 0u;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) acc[j] += c * (int64_t)a0[j] - (int64_t)a1[j];
  }
}

template <int T>
__device__ __noinline__ void fs1_list_wide(const uint32_t *s, int beg, int end, const int64_t (&lam)[T], int64_t c,
                          int64_t (&acc)[T]) {
  for (int i = beg; i < end; ++i) {
    const int64_t w = s[i];
#pragma unroll
    for (int j = 0; j < T; ++j) {
      const int64_t x = w * (lam[j] + 1);
      acc[j] += c * (x / c) - ((x % c == 0) ? w : 0);
    }
  }
}

// ---- CCM1 (u2 = 2u): acc += SIGN * floor(u / l) ---------------------------------
template <int T, int SIGN>
BPLB_D void ccm1_list(const uint32_t *s, int beg, int end, int K, const Div31 (&D)[T],
                      int64_t (&acc)[T]) {
  for (int g0 = beg; g0 < end; g0 += K) {
    const int g1 = min(end, g0 + K);
    uint32_t a[T];
#pragma unroll
    for (int j = 0; j < T; ++j) a[j] = 0;
#pragma unroll 2
    for (int i = g0; i < g1; i += 4) {
      const uint4 v = lds4(s, i);
#pragma unroll
      for (int j = 0; j < T; ++j) {
        a[j] += div31(v.x, D[j]) + div31(v.y, D[j]);
        a[j] += div31(v.z, D[j]) + div31(v.w, D[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) acc[j] += SIGN * (int64_t)a[j];
  }
}

// mad.hi.u32: hi32(a * b) + c in one integer multiply-add (FMA pipe).
BPLB_D uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// c <= 131071, list holds u (not 2u): acc += SIGN * floor(u / l) with one
// multiply-high-add per item (no shift; u * l < 2^32).  For l = 1 each nonzero
// item yields u - 1: the caller adds the item count back.
template <int T, int SIGN>
BPLB_D void ccm1_list_noshift(const uint32_t *s, int beg, int end, int K, const uint32_t (&m1)[T],
                              int64_t (&acc)[T]) {
  for (int g0 = beg; g0 < end; g0 += K) {
    const int g1 = min(end, g0 + K);
    uint32_t a[T];
#pragma unroll
    for (int j = 0; j < T; ++j) a[j] = 0;
#pragma unroll 2
    for (int i = g0; i < g1; i += 4) {
      const uint4 v = lds4(s, i);
#pragma unroll
      for (int j = 0; j < T; ++j) {
        a[j] = mad_hi(v.x, m1[j], a[j]);
        a[j] = mad_hi(v.y, m1[j], a[j]);
        a[j] = mad_hi(v.z, m1[j], a[j]);
        a[j] = mad_hi(v.w, m1[j], a[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) acc[j] += SIGN * (int64_t)a[j];
  }
}

// ---- VB2, c <= 65535: acc += SIGN * sum ceil(u l / c) by fixed-point fractions ----
// The list holds F = ceil(u 2^32 / c) (< 2^31 as u < c / 2).  With
// Y0 = ceil((c - 1) 2^32 / c), the 64-bit Y = l F + Y0 equals
// 2^32 (u l + c - 1) / c + e with 0 <= e < l + 1; the fraction of
// (u l + c - 1) / c is at most (c - 1) / c, and (l + 1) c < 2^32 keeps
// e / 2^32 below 1 / c, so floor(Y / 2^32) = floor((u l + c - 1) / c)
// = ceil(u l / c) exactly.  Over a list of n entries,
//   sum floor(Y / 2^32) = (sum Y - Z) / 2^32,  Z = sum (Y mod 2^32),
// with sum Y = l sum F + n Y0 known and Y mod 2^32 one 32-bit multiply-add
// per item: no multiply-high in the loop.  Z itself is not summed: with
// H = sum ((Y mod 2^32) >> 16) (a 32-bit sum while n < 2^16),
// Z lies in [H 2^16, H 2^16 + n 2^16) and Z = sum Y mod 2^32, so
//   sum floor(Y / 2^32) = (sum Y - H 2^16) >> 32.
// Padding slots hold F = 0 and cancel.
template <int T, int SIGN>
BPLB_D void vb2_list_fixed(const uint32_t *s, int beg, int end, const uint32_t (&lam)[T],
                           uint32_t Y0, uint64_t sumF, int64_t (&acc)[T]) {
  uint32_t h[T];
#pragma unroll
  for (int j = 0; j < T; ++j) h[j] = 0;
#pragma unroll 2
  for (int i = beg; i < end; i += 4) {
    const uint4 v = lds4(s, i);
#pragma unroll
    for (int j = 0; j < T; ++j) {
      h[j] += ((v.x * lam[j] + Y0) >> 16) + ((v.y * lam[j] + Y0) >> 16);
      h[j] += ((v.z * lam[j] + Y0) >> 16) + ((v.w * lam[j] + Y0) >> 16);
    }
  }
  const uint64_t nY0 = (uint64_t)(end - beg) * Y0;
#pragma unroll
  for (int j = 0; j < T; ++j)
    acc[j] += SIGN * (int64_t)(((uint64_t)lam[j] * sumF + nY0 - ((uint64_t)h[j] << 16)) >> 32);
}

// The fixed-point list value F = ceil(u 2^32 / c) and offset Y0 of vb2_list_fixed.
BPLB_HD uint32_t vb2_fixed_frac(uint64_t u, uint64_t c) { return (uint32_t)(((u << 32) + c - 1) / c); }

// 65535 < c <= 2^22: an fp32 estimate of the quotient, corrected exactly.
//   a = fl(u / c) (correctly rounded, staged with the list), relative error
//   <= 2^-24.  fmaf(l, a, 1.5 * 2^23) rounds l*a + 1.5*2^23 to an integer
//   since the sum lies in [2^23, 2^24); its bit pattern is 0x4B400000 + q~
//   with q~ = round(l * a), and |q~ - u l / c| <= 1/2 + (c/2) 2^-24 < 1.
//   The residual 2 rho = u2 l - 2c q~ is then in (-2c, 2c), so it is exact in
//   wrapping 32-bit arithmetic, and ceil(u l / c) = q~ + [rho > 0].
//   The loop accumulates bits + [rho > 0] modulo 2^32 and removes
//   0x4B400000 per list slot at the end of each group.
constexpr uint32_t kF32RoundBits = 0x4B400000u;  // bit pattern of 1.5 * 2^23

template <int T, int SIGN>
BPLB_D void vb2_list_float(const uint32_t *s, const float *sa, int beg, int end, int K,
                           const uint32_t (&lam)[T], const float (&lamf)[T], uint32_t c2,
                           uint32_t K2, int64_t (&acc)[T]) {
  for (int g0 = beg; g0 < end; g0 += K) {
    const int g1 = min(end, g0 + K);
    uint32_t a[T];
#pragma unroll
    for (int j = 0; j < T; ++j) a[j] = 0;
#pragma unroll 2
    for (int i = g0; i < g1; i += 4) {
      const uint4 v = lds4(s, i);
      const float4 f = lds4f(sa, i);
      const uint32_t u4[4] = {v.x, v.y, v.z, v.w};
      const float f4[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
          const uint32_t bits = __float_as_uint(__fmaf_rn(lamf[j], f4[e], 12582912.0f));
          const uint32_t neg2rho = bits * c2 + K2 - u4[e] * lam[j];  // = -2 rho (mod 2^32)
          a[j] += bits + (neg2rho >> 31);
        }
      }
    }
    const uint32_t slots = (uint32_t)(g1 - g0);
#pragma unroll
    for (int j = 0; j < T; ++j) acc[j] += SIGN * (int64_t)(uint32_t)(a[j] - slots * kF32RoundBits);
  }
}

template <int T, int SIGN>
__device__ __noinline__ void vb2_list_wide(const uint32_t *s, int beg, int end, const int64_t (&lam)[T], int64_t c,
                          int64_t (&acc)[T]) {
  for (int i = beg; i < end; ++i) {
    const int64_t u = s[i] >> 1;
#pragma unroll
    for (int j = 0; j < T; ++j) acc[j] += SIGN * ((u * lam[j] + c - 1) / c);
  }
}

// ---- BJ1 (w2 = 2w): acc += cm * floor(w / l) + min(w mod l, cm) ---------------
template <int T>
BPLB_D void bj1_list(const uint32_t *s, int beg, int end, int K, const Div31 (&D)[T],
                     const uint32_t (&l2)[T], const uint32_t (&cm2)[T], int64_t (&acc)[T]) {
  for (int g0 = beg; g0 < end; g0 += K) {
    const int g1 = min(end, g0 + K);
    uint32_t a0[T], a1[T];
#pragma unroll
    for (int j = 0; j < T; ++j) a0[j] = a1[j] = 0;
#pragma unroll 2
    for (int i = g0; i < g1; i += 4) {
      const uint4 v = lds4(s, i);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
          const uint32_t q = div31(w4[e], D[j]);
          const uint32_t r2 = w4[e] - q * l2[j];  // 2 (w mod l)
          a0[j] += q;
          a1[j] += min(r2, cm2[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < T; ++j)
      acc[j] += (int64_t)(cm2[j] >> 1) * (int64_t)a0[j] + (int64_t)(a1[j] >> 1);
  }
}

// c <= 65535, list holds raw w: q = floor(w / l) by multiply-high without a
// shift (w * l < 2^32), rho = w - q l; acc += cm * sum q + sum min(rho, cm)
// with cm = c mod l: two multiply-adds (FMA pipe) and a min plus two adds (ALU
// pipe) per item.  For l = 1, cm = 0 and q (= w - 1 for w >= 1) is multiplied
// by 0, min(rho, 0) = 0: the term is 0, as it must be.
template <int T>
BPLB_D void bj1_list_noshift(const uint32_t *s, int beg, int end, int K, const uint32_t (&m1)[T],
                             const uint32_t (&lam)[T], const uint32_t (&cm)[T],
                             int64_t (&acc)[T]) {
  for (int g0 = beg; g0 < end; g0 += K) {
    const int g1 = min(end, g0 + K);
    uint32_t a0[T], a1[T];
#pragma unroll
    for (int j = 0; j < T; ++j) a0[j] = a1[j] = 0;
#pragma unroll 2
    for (int i = g0; i < g1; i += 4) {
      const uint4 v = lds4(s, i);
      const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
#pragma unroll
        for (int j = 0; j < T; ++j) {
          const uint32_t q = __umulhi(w4[e], m1[j]);
          a0[j] += q;
          a1[j] += min(w4[e] - q * lam[j], cm[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < T; ++j) acc[j] += (int64_t)cm[j] * (int64_t)a0[j] + (int64_t)a1[j];
  }
}

template <int T>
__device__ __noinline__ void bj1_list_wide(const uint32_t *s, int beg, int end, const int64_t (&lam)[T], int64_t c,
                          int64_t (&acc)[T]) {
  for (int i = beg; i < end; ++i) {
    const int64_t w = s[i] >> 1;
#pragma unroll
    for (int j = 0; j < T; ++j) {
      const int64_t q = w / lam[j], rho = w % lam[j], cm = c % lam[j];
      acc[j] += cm * q + (rho < cm ? rho : cm);
    }
  }
}

}  // namespace bplb
