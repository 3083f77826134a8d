// Instantiates eval_kernel for every launch shape of bp_lb_launch.cuh, input
// mode kSrcRaggedI64.
#include "bp_lb_launch.cuh"

BPLB_INSTANTIATE_MODE(eval_fn_ragged_i64, kSrcRaggedI64)
