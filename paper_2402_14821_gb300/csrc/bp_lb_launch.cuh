// bp_lb_launch.cuh -- the table of compiled launch shapes of eval_kernel.
//
// Each shape is (NT threads per CTA, T parameters per thread per group, G
// groups per tile, MINB resident CTAs per SM -- which caps registers at
// 65536 / (NT * MINB)) of the generic direct kernel, and VT, the parameters
// per thread of the VB2 kernel launched with it.  Every shape is instantiated
// for the three input modes in its own translation unit
// (bp_lb_inst_<mode>.cu) and picked at run time per handle, by default or by
// the autotuner.
#pragma once

#include <cuda_runtime.h>

#include "bp_lb_kernels.cuh"
#include "bp_lb_cluster.cuh"
#include "bp_lb_prefix.cuh"
#include "bp_lb_vb2.cuh"

namespace bplb {

struct LaunchShape {
  int nt, t, g, minb, vt;
};

constexpr int kNumShapes = 8;
constexpr LaunchShape kShapes[kNumShapes] = {
    {256, 4, 2, 3, 4},  // 0: default
    {256, 2, 4, 4, 8},  // 1: fewer registers, more resident warps
    {128, 4, 2, 6, 2},  // 2: smaller CTAs
    {256, 4, 4, 3, 8},  // 3: longer tiles (less staging per parameter)
    {128, 4, 4, 6, 4},  // 4: small CTAs, longer tiles
    {128, 4, 8, 6, 4},  // 5: small CTAs, longest tiles (search nodes)
    {128, 2, 1, 6, 2},  // 6: short tiles: one check spread over all SMs (latency)
    {128, 1, 1, 8, 8},  // 7: shortest tiles (latency)
};

constexpr int64_t shape_lpt(int s) { return (int64_t)kShapes[s].nt * kShapes[s].t * kShapes[s].g; }

using EvalFn = void (*)(EvalArgs);

// Host stubs of the instantiated kernels, one table per input mode; shape -1
// is the prefix-count kernel of that mode, shape -2 - s the VB2 kernel with
// shape s's VT, kClusterShape the cluster kernel.
EvalFn eval_fn_ragged_i32(int shape);
EvalFn eval_fn_ragged_i64(int shape);
EvalFn eval_fn_nodes(int shape);

inline EvalFn eval_fn(int shape, int mode) {
  switch (mode) {
    case kSrcRaggedI32: return eval_fn_ragged_i32(shape);
    case kSrcRaggedI64: return eval_fn_ragged_i64(shape);
    default: return eval_fn_nodes(shape);
  }
}

constexpr int kClusterShape = -1000;

inline EvalFn prefix_fn(int mode) { return eval_fn(-1, mode); }
inline EvalFn cluster_fn(int mode) { return eval_fn(kClusterShape, mode); }
inline EvalFn vb2_fn(int shape, int mode) { return eval_fn(-2 - shape, mode); }

}  // namespace bplb

// Instantiates every shape of one mode (used once per translation unit).
#define BPLB_INSTANTIATE_MODE(NAME, MODE)                                          \
  namespace bplb {                                                                 \
  EvalFn NAME(int shape) {                                                         \
    if (shape == kClusterShape) return cluster_kernel<MODE>;                       \
    if (shape <= -2) {                                                             \
      switch (kShapes[-2 - shape].vt) {                                            \
        case 2: return vb2_kernel<MODE, 2>;                                        \
        case 4: return vb2_kernel<MODE, 4>;                                        \
        default: return vb2_kernel<MODE, 8>;                                       \
      }                                                                            \
    }                                                                              \
    switch (shape) {                                                               \
      case -1: return prefix_kernel<MODE>;                                         \
      case 0: return eval_kernel<kShapes[0].nt, kShapes[0].t, kShapes[0].g, MODE,  \
                                 kShapes[0].minb>;                                 \
      case 1: return eval_kernel<kShapes[1].nt, kShapes[1].t, kShapes[1].g, MODE,  \
                                 kShapes[1].minb>;                                 \
      case 2: return eval_kernel<kShapes[2].nt, kShapes[2].t, kShapes[2].g, MODE,  \
                                 kShapes[2].minb>;                                 \
      case 3: return eval_kernel<kShapes[3].nt, kShapes[3].t, kShapes[3].g, MODE,  \
                                 kShapes[3].minb>;                                 \
      case 4: return eval_kernel<kShapes[4].nt, kShapes[4].t, kShapes[4].g, MODE,  \
                                 kShapes[4].minb>;                                 \
      case 5: return eval_kernel<kShapes[5].nt, kShapes[5].t, kShapes[5].g, MODE,  \
                                 kShapes[5].minb>;                                 \
      case 6: return eval_kernel<kShapes[6].nt, kShapes[6].t, kShapes[6].g, MODE,  \
                                 kShapes[6].minb>;                                 \
      default: return eval_kernel<kShapes[7].nt, kShapes[7].t, kShapes[7].g, MODE, \
                                  kShapes[7].minb>;                                \
    }                                                                              \
  }                                                                                \
  }
