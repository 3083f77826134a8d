// bp_lb_vb2.cuh -- the VB2 kernel: VB2 on its fixed-point path (c <= 65535).
//
// VB2 has about c parameters, more than any other DFF except BJ1, and no
// prefix-count form (its breakpoints c j / l move with every l), so in a
// batch it is most of the item-by-item work.  Its fixed-point evaluator
// (vb2_list_fixed: one 32-bit multiply-add and half of a two-word add per
// item and parameter) needs few registers; in the generic direct kernel it
// would run at the occupancy that kernel's widest DFF path allows.  This
// kernel evaluates the VB2 tiles alone, with the same tile evaluation
// (tile_dff) compiled for VB2's fixed-point path only, so that its register
// footprint -- and hence its resident warps -- are VB2's own.  Tiles carry
// vlpt consecutive parameters of one instance (the plan kernel's choice,
// kVb2LPT at least); finalisation is shared with
// the other kernels through the instance's key slot and finished-tile ticket.
#pragma once

#include "bp_lb_kernels.cuh"

namespace bplb {

constexpr int kVb2NT = 128;

// Resident CTAs per SM asked of the compiler for VT parameters per thread
// (registers capped at 65536 / (128 MINB)).
constexpr int vb2_minb(int vt) { return vt <= 2 ? 10 : (vt <= 4 ? 8 : 6); }

// Dynamic shared memory: the two item lists, then the bin loads of a node.
constexpr size_t kVb2ListBytes = sizeof(uint32_t) * kListTop;

template <int MODE, int VT>
__global__ void __launch_bounds__(kVb2NT, vb2_minb(VT)) vb2_kernel(EvalArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ TileShared S;
  __shared__ TileCursor cur;
  uint32_t *s_items = reinterpret_cast<uint32_t *>(smem_raw);
  uint32_t *s_load = reinterpret_cast<uint32_t *>(smem_raw + kVb2ListBytes);

  pdl_wait();
  pdl_release();
  const int64_t total = A.vtile_start ? A.vtile_start[A.B] : A.single_vtiles;
  const int64_t vlpt = A.vlpt != nullptr ? (int64_t)*A.vlpt : kVb2LPT;
  work_count_begin(A, S);
  tile_first(A.vtile_start, A.B, total, A.vwork, cur);
  while (cur.tile < total) {
    const int64_t t = cur.tile, b = cur.inst;
    const unsigned long long next = tile_claim(A.vwork);
    // VB2 already evaluated on the instance's u-group tile (its sums flag
    // 2): the tile only counts itself, with nothing to fold and without the
    // instance's fields unless it is the instance's last
    if (threadIdx.x == 0)
      S.done_vb2 = A.isums != nullptr && (A.verdict || A.prune) &&
                   reinterpret_cast<const volatile long long *>(A.isums)[8 * b + 7] == 2;
    __syncthreads();
    if (S.done_vb2) {
      if (threadIdx.x == 32) {  // fold_and_finalize's thread, best key 0
        __threadfence();
        const int64_t ntiles = instance_tiles(A, b);
        const unsigned int ticket = atomicAdd(&A.done[b], 1u);
        if (ntiles > 0 ? (int64_t)ticket == ntiles - 1 : ticket == 0xFFFFFFFFu) {
          __threadfence();
          const unsigned long long key = atomicExch(&A.keys[b], 0ull);
          A.done[b] = 0u;
          const InstView I = resolve_instance<MODE>(A, b);
          write_result(A, b, key, I.c, I.k);
        }
      }
      if (!A.vwork) break;
      tile_publish(A.vtile_start, A.B, total, next, cur);
      continue;
    }
    const InstView I = resolve_instance<MODE>(A, b);
    const int64_t t0 = A.vtile_start ? A.vtile_start[b] : 0;
    const int64_t ntiles = instance_tiles(A, b);
    int64_t lo_d, hi_d;
    param_range(kVB2, I.c, lo_d, hi_d);
    hi_d = vb2_last(A, b, hi_d);  // the cap of Sec. 4, when on
    const int64_t lam0 = lo_d + (t - t0) * vlpt;
    const int64_t lam_end = max(lam0, min(hi_d + 1, lam0 + vlpt));

    unsigned long long *vslot = A.verdict ? &A.keys[b] : nullptr;
    if (threadIdx.x == 0) {
      S.err = 0;
      S.skip = ((vslot != nullptr && slot_decided(vslot, I.k)) || lam_end <= lam0) ? 1 : 0;
      // the whole tile pruned (vb2_range_may_exceed) from the instance sums the
      // prefix kernel published, before anything is staged
      if (!S.skip && A.isums != nullptr && (A.verdict || A.prune)) {
        const volatile long long *is = A.isums + 8 * b;
        const long long flag = is[7];
        if (flag == 2) S.skip = 1;  // VB2 done on the u-group tile since the check above
        if (flag == 1) {
          __threadfence();
          const int64_t cut = A.verdict ? I.k : (int64_t)vb2_cut(&A.keys[b], flat_index(kVB2, lo_d, I.c));
          if (cut >= 0) {
            const int64_t c = I.c;
            const int64_t ns = is[0], nb = is[1], nh = is[2], nf = is[3], swb = is[4], sw = is[5];
            const int64_t Dd = (sw - swb - nh * (c / 2) - nf * c) - (nb * c - swb);
            const int64_t K = 2 * nb + nh + 2 * nf;
            const int64_t kk = min(cut, stream_len<MODE>(I));
            if (!vb2_range_may_exceed(lam0, lam_end - 1, kk, c, Dd, ns, nb, K)) {
              S.skip = 1;
              if (A.work_count != nullptr) atomicAdd(&S.wc[3], (unsigned long long)(lam_end - lam0));
            }
          }
        }
      }
    }
    __syncthreads();
    unsigned long long best = 0ull;
    if (!S.skip) {
      node_loads<kVb2NT, MODE>(A, b, I, s_load, &S.minw, &S.err);
      __syncthreads();
      best = tile_dff<kVb2NT, VT, kVB2, MODE, false, true>(
          A, I, lam0, lam_end, s_items, nullptr, s_load, S, nullptr, nullptr, -1, vslot,
          A.prune && !A.verdict ? &A.keys[b] : nullptr);
    }
    __syncthreads();
    fold_and_finalize<kVb2NT>(A, b, best, S.err != 0, ntiles, I, S.warp_key);
    if (!A.vwork) break;
    tile_publish(A.vtile_start, A.B, total, next, cur);
  }
  work_count_flush(A, S);
}

}  // namespace bplb
