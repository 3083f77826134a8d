// Instantiates eval_kernel for every launch shape of bp_lb_launch.cuh, input
// mode kSrcNodes.
#include "bp_lb_launch.cuh"

BPLB_INSTANTIATE_MODE(eval_fn_nodes, kSrcNodes)
