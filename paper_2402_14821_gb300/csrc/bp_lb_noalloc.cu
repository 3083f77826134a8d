// bp_lb_noalloc.cu -- bp_lb_eval_batch_noalloc: the batched check over ragged
// int32 instances without a handle and without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// check -- code whose device memory is owned entirely by another allocator
// (a framework's caching pool that has reserved the whole device), search
// loops that must not pay the device-wide synchronisation cudaFree implies
// between their own kernels, and embedded solvers that fix their device memory
// budget at start-up.  bp_lb_create allocates staging and scratch, so those
// callers use this entry point instead.
//
// The scratch the planning and evaluation kernels need (work counter, tile
// table, per-instance result slots and finished-tile counters) lives in one
// file-scope __device__ array of fixed size, sized for at most
// BP_NOALLOC_MAX_BATCH instances.  Every GPU that loads the library holds that
// array until the process exits.  Host code cannot use the array's name as a
// device address (on the host it names a host-side shadow), so the device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, and passed to the kernels.
//
// It evaluates every DFF item by item in the generic kernel (the direct
// algorithm, with VB2 there too, launch shape 0): the prefix-count tables and
// the VB2 kernel need per-call scratch that only a handle owns.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/bp_lb.h"
#include "bp_lb_kernels.cuh"
#include "bp_lb_launch.cuh"

using namespace bplb;

namespace {

constexpr int64_t kNoAllocMax = BP_NOALLOC_MAX_BATCH;
// Layout (byte offsets, each 256-aligned): work counter, tile table
// [kNoAllocMax + 1], result slots [kNoAllocMax], finished-tile counters
// [kNoAllocMax].
constexpr size_t kOffWork = 0;
constexpr size_t kOffTiles = 256;
constexpr size_t kOffKeys = kOffTiles + ((sizeof(int64_t) * (kNoAllocMax + 1) + 255) / 256) * 256;
constexpr size_t kOffDone = kOffKeys + ((sizeof(unsigned long long) * kNoAllocMax + 255) / 256) * 256;
constexpr size_t kScratchBytes = kOffDone + ((sizeof(unsigned int) * kNoAllocMax + 255) / 256) * 256;

constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_noalloc_mu;

// Per-device set-up, done once with that device current: the array's device
// address, the evaluation kernel's resident CTAs per SM and the SM count.
struct NoAllocDevice {
  void *addr = nullptr;
  int sms = 0;
  int occ = 0;
};
NoAllocDevice g_noalloc_dev[kMaxDevices];

constexpr int kNoAllocShape = 0;
constexpr size_t kNoAllocSmem = 2 * sizeof(uint32_t) * kListTop;

// The current device's set-up, done on its first call: looks up the device
// address of g_noalloc_scratch (cudaGetSymbolAddress) and queries the two
// kernels this entry point launches (which loads them, and the array, under
// CUDA's lazy module loading), so that later calls only launch.
int noalloc_setup(NoAllocDevice *out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BP_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return BP_ERANGE;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice &d = g_noalloc_dev[dev];
  if (!d.addr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BP_ECUDA;
    cudaFuncAttributes fa;
    const void *fn = (const void *)eval_fn(kNoAllocShape, kSrcRaggedI32);
    int sms = 0, occ = 0;
    if (cudaFuncGetAttributes(&fa, (const void *)plan_kernel<kSrcRaggedI32>) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kShapes[kNoAllocShape].nt,
                                                      kNoAllocSmem) != cudaSuccess ||
        occ <= 0)
      return BP_ECUDA;
    d.sms = sms;
    d.occ = occ;
    d.addr = p;
  }
  *out = d;
  return BP_OK;
}

}  // namespace

extern "C" int bp_lb_eval_batch_noalloc(int32_t B, const int64_t *d_offsets,
                                        const int32_t *d_sizes, const int64_t *d_capacity,
                                        const int64_t *d_bins, int64_t *d_out_bound,
                                        bp_argmax_t *d_out_argmax, uint8_t *d_out_feasible,
                                        void *stream) {
  if (B < 0) return BP_EINVAL;
  if (B > kNoAllocMax) return BP_ERANGE;
  // the per-device set-up runs on the first call, B = 0 included
  NoAllocDevice nd;
  const int st = noalloc_setup(&nd);
  if (st != BP_OK) return st;
  if (B == 0) return BP_OK;
  if (!d_offsets || !d_sizes || !d_capacity || !d_bins || !d_out_bound) return BP_EINVAL;
  unsigned char *scratch = static_cast<unsigned char *>(nd.addr);

  EvalArgs A;
  std::memset(&A, 0, sizeof(A));
  A.one = 1u;
  A.prune = 1;
  A.B = B;
  A.offsets = d_offsets;
  A.sizes = d_sizes;
  A.capacity = d_capacity;
  A.bins = d_bins;
  A.out_bound = d_out_bound;
  A.out_argmax = d_out_argmax;
  A.out_feasible = d_out_feasible;
  A.work = reinterpret_cast<unsigned long long *>(scratch + kOffWork);
  A.tile_start = reinterpret_cast<const int64_t *>(scratch + kOffTiles);
  A.keys = reinterpret_cast<unsigned long long *>(scratch + kOffKeys);
  A.done = reinterpret_cast<unsigned int *>(scratch + kOffDone);

  const int shape = kNoAllocShape;
  const void *fn = (const void *)eval_fn(shape, kSrcRaggedI32);
  cudaStream_t s = (cudaStream_t)stream;
  // The planning kernel clears the result slots, finished-tile counters and
  // work counter of the B instances before the evaluation kernel runs.
  plan_kernel<kSrcRaggedI32><<<1, 1024, 0, s>>>(A, shape_lpt(shape),
                                                reinterpret_cast<int64_t *>(scratch + kOffTiles),
                                                nullptr, nullptr, nullptr);
  if (cudaGetLastError() != cudaSuccess) return BP_ECUDA;
  void *args[] = {&A};
  if (cudaLaunchKernel(fn, dim3((unsigned)(nd.sms * nd.occ)), dim3(kShapes[shape].nt), args,
                       kNoAllocSmem, s) != cudaSuccess)
    return BP_ECUDA;
  return BP_OK;
}
