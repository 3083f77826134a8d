// bp_lb_probe.cu -- measurement aid: the integer instruction issue rate of the
// device, the denominator of the item-by-item kernels' roofline.
//
// The item-by-item DFF evaluators are bound by integer instruction issue: a
// sub-partition issues at most one warp instruction per clock, and integer
// multiply-adds (FMA pipe) and logic/add/shift/compare (ALU pipe) each run at
// half that rate, so only a mix of the two can reach it.  The probe kernel
// runs exactly such a mix with no memory traffic: per thread eight
// independent chains, each step one multiply-add a = a * K + b and one xor
// b ^= a, unrolled sixteen steps deep; timing one launch with CUDA events gives
// the lane operations per second the device sustains at its current clock.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/bp_lb.h"

namespace {

constexpr int kProbeNT = 256;
constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;
// integer operations per thread and loop trip: chains x unroll x (mul-add + xor)
constexpr int64_t kProbeOpsPerTrip = kProbeChains * kProbeUnroll * 2;

__global__ void __launch_bounds__(kProbeNT) int_issue_probe(uint32_t *sink, int32_t trips,
                                                             uint32_t seed) {
  uint32_t a[kProbeChains], b[kProbeChains];
  const uint32_t t = blockIdx.x * kProbeNT + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) {
    a[j] = seed ^ (t * 2654435761u + (uint32_t)j);
    b[j] = seed + t + 977u * (uint32_t)j;
  }
  for (int32_t i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kProbeChains; ++j) {
        a[j] = a[j] * 0x9E3779B1u + b[j];
        b[j] ^= a[j];
      }
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) x ^= a[j] + b[j];
  sink[t] = x;  // keeps the chains live
}

}  // namespace

extern "C" int bp_lb_probe_int_issue(int32_t blocks_per_sm, int32_t trips, uint32_t *d_sink,
                                     void *stream, int64_t *out_lane_ops) {
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || trips < 1 || !d_sink || !out_lane_ops)
    return BP_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return BP_ECUDA;
  const unsigned grid = (unsigned)(sms * blocks_per_sm);
  int_issue_probe<<<grid, kProbeNT, 0, (cudaStream_t)stream>>>(d_sink, trips, 0x2545F491u);
  if (cudaGetLastError() != cudaSuccess) return BP_ECUDA;
  *out_lane_ops = (int64_t)grid * kProbeNT * (int64_t)trips * kProbeOpsPerTrip;
  return BP_OK;
}
