// bp_serve.cu -- continuous-batching request loop for feasibility checks
// (include/bp_lb.h, "serving").
//
// Searches register their base instances once (the sizes stay resident in a
// device pool) and then submit checks: a partial packing (one bin index or -1
// per item) and a bin count.  A scheduler thread forms batches from the
// pending requests whenever one of its in-flight slots is free, copies the
// batch's assignments host->device, and runs the fused reduction + bound
// evaluation (bp_lb_eval_nodes) on that slot's stream.  Each slot has its own
// handle (scratch), stream and staging, so a batch admitted while others are
// still on the GPU runs concurrently with them: its CTAs start as the earlier
// batches' CTAs retire.  Admission is by device-memory footprint: the resident
// pool has a fixed size, and pending + in-flight assignment bytes are bounded;
// a request that does not fit is refused with BP_EBUSY (the caller retries).
//
// All waits are bounded (condition-variable waits with timeouts and CUDA
// event queries); nothing spins on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/bp_lb.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  int64_t tag;
  int32_t instance;
  int64_t bins;
  std::vector<int32_t> assign;
  Clock::time_point t_submit;
};

struct Slot {
  bp_lb_t *h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  // staging (pinned host) and device copies of one batch
  int32_t *h_assign = nullptr, *d_assign = nullptr;
  int64_t *h_aoff = nullptr, *d_aoff = nullptr;
  int32_t *h_base = nullptr, *d_base = nullptr;
  int64_t *h_bins = nullptr, *d_bins = nullptr;
  int64_t *h_bound = nullptr, *d_bound = nullptr;
  bp_argmax_t *h_arg = nullptr, *d_arg = nullptr;
  uint8_t *h_feas = nullptr, *d_feas = nullptr;
  std::vector<Request> batch;
  bool failed = false;  // the launch of `batch` failed: report BP_ECUDA
};

}  // namespace

struct bp_serve {
  // configuration
  int64_t pool_items = 0;
  int32_t max_instances = 0;
  int64_t max_queued_items = 0;
  int32_t max_batch = 0;
  int64_t slot_items = 0;
  int64_t max_bins = 0;
  int device = 0;
  // resident instance pool
  int32_t *d_pool = nullptr;
  int64_t *d_pool_off = nullptr;   // [max_instances + 1]
  int64_t *d_pool_cap = nullptr;   // [max_instances]
  std::vector<int64_t> pool_off;   // host mirror
  std::vector<int64_t> pool_cap;
  int32_t n_instances = 0;
  // requests
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> pending;
  int64_t queued_items = 0;        // pending + in flight
  int64_t next_id = 1;
  std::vector<bp_serve_result_t> completed;
  std::vector<Slot> slots;
  std::thread worker;
  std::atomic<bool> stop{false};
  int worker_status = BP_OK;
  // statistics
  int64_t n_batches = 0, n_done = 0, n_refused = 0;
};

namespace {

int cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return BP_OK;
  if (e == cudaErrorMemoryAllocation) return BP_ENOMEM;
  return BP_ECUDA;
}

void free_slot(Slot &s) {
  if (s.h) bp_lb_destroy(s.h);
  if (s.stream) cudaStreamDestroy(s.stream);
  if (s.done) cudaEventDestroy(s.done);
  cudaFreeHost(s.h_assign);
  cudaFreeHost(s.h_aoff);
  cudaFreeHost(s.h_base);
  cudaFreeHost(s.h_bins);
  cudaFreeHost(s.h_bound);
  cudaFreeHost(s.h_arg);
  cudaFreeHost(s.h_feas);
  cudaFree(s.d_assign);
  cudaFree(s.d_aoff);
  cudaFree(s.d_base);
  cudaFree(s.d_bins);
  cudaFree(s.d_bound);
  cudaFree(s.d_arg);
  cudaFree(s.d_feas);
  s = Slot();
}

int alloc_slot(Slot &s, int64_t items, int32_t max_batch) {
  int st = bp_lb_create(1, 1, &s.h);
  if (st != BP_OK) return st;
  if ((st = bp_lb_reserve(s.h, max_batch)) != BP_OK) return st;
  if ((st = cuda_st(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking))) != BP_OK) return st;
  if ((st = cuda_st(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming))) != BP_OK) return st;
  const size_t B = (size_t)max_batch;
#define BPS_ALLOC(hp, dp, count)                                                       \
  if ((st = cuda_st(cudaMallocHost(&(hp), sizeof(*(hp)) * (count)))) != BP_OK) return st; \
  if ((st = cuda_st(cudaMalloc(&(dp), sizeof(*(dp)) * (count)))) != BP_OK) return st;
  BPS_ALLOC(s.h_assign, s.d_assign, (size_t)items)
  BPS_ALLOC(s.h_aoff, s.d_aoff, B + 1)
  BPS_ALLOC(s.h_base, s.d_base, B)
  BPS_ALLOC(s.h_bins, s.d_bins, B)
  BPS_ALLOC(s.h_bound, s.d_bound, B)
  BPS_ALLOC(s.h_arg, s.d_arg, B)
  BPS_ALLOC(s.h_feas, s.d_feas, B)
#undef BPS_ALLOC
  return BP_OK;
}

// Launches the slot's batch (called with the server lock released).
int launch_slot(bp_serve *S, Slot &s, int32_t n_inst) {
  const int32_t B = (int32_t)s.batch.size();
  int64_t off = 0;
  for (int32_t b = 0; b < B; ++b) {
    const Request &r = s.batch[b];
    s.h_aoff[b] = off;
    std::memcpy(s.h_assign + off, r.assign.data(), sizeof(int32_t) * r.assign.size());
    off += (int64_t)r.assign.size();
    s.h_base[b] = r.instance;
    s.h_bins[b] = r.bins;
  }
  s.h_aoff[B] = off;
  int st = BP_OK;
  if (off > 0 &&
      (st = cuda_st(cudaMemcpyAsync(s.d_assign, s.h_assign, sizeof(int32_t) * off,
                                    cudaMemcpyHostToDevice, s.stream))) != BP_OK)
    return st;
  if ((st = cuda_st(cudaMemcpyAsync(s.d_aoff, s.h_aoff, sizeof(int64_t) * (B + 1),
                                    cudaMemcpyHostToDevice, s.stream))) != BP_OK)
    return st;
  if ((st = cuda_st(cudaMemcpyAsync(s.d_base, s.h_base, sizeof(int32_t) * B,
                                    cudaMemcpyHostToDevice, s.stream))) != BP_OK)
    return st;
  if ((st = cuda_st(cudaMemcpyAsync(s.d_bins, s.h_bins, sizeof(int64_t) * B,
                                    cudaMemcpyHostToDevice, s.stream))) != BP_OK)
    return st;
  st = bp_lb_eval_nodes(s.h, B, n_inst, S->d_pool_off, S->d_pool, S->d_pool_cap, s.d_base,
                        s.d_aoff, s.d_assign, s.d_bins, S->max_bins, s.d_bound, s.d_arg, s.d_feas,
                        s.stream);
  if (st != BP_OK) return st;
  if ((st = cuda_st(cudaMemcpyAsync(s.h_bound, s.d_bound, sizeof(int64_t) * B,
                                    cudaMemcpyDeviceToHost, s.stream))) != BP_OK)
    return st;
  if ((st = cuda_st(cudaMemcpyAsync(s.h_arg, s.d_arg, sizeof(bp_argmax_t) * B,
                                    cudaMemcpyDeviceToHost, s.stream))) != BP_OK)
    return st;
  if ((st = cuda_st(cudaMemcpyAsync(s.h_feas, s.d_feas, sizeof(uint8_t) * B,
                                    cudaMemcpyDeviceToHost, s.stream))) != BP_OK)
    return st;
  return cuda_st(cudaEventRecord(s.done, s.stream));
}

// The scheduler: collects finished slots, then fills free slots from the
// pending queue (FIFO, up to max_batch requests and slot_items assignment
// entries per batch).
void worker_loop(bp_serve *S) {
  cudaSetDevice(S->device);
  while (true) {
    bool did = false;
    // 1. finished batches
    for (Slot &s : S->slots) {
      if (!s.busy) continue;
      const cudaError_t q = s.failed ? cudaErrorUnknown : cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      const auto now = Clock::now();
      std::lock_guard<std::mutex> lock(S->mu);
      const int err = (q == cudaSuccess) ? BP_OK : BP_ECUDA;
      for (size_t b = 0; b < s.batch.size(); ++b) {
        const Request &r = s.batch[b];
        bp_serve_result_t res;
        std::memset(&res, 0, sizeof(res));
        res.request = r.id;
        res.tag = r.tag;
        res.bound = err ? -BP_ECUDA : s.h_bound[b];
        res.argmax = s.h_arg[b];
        res.feasible = err ? 0 : s.h_feas[b];
        res.status = err ? BP_ECUDA : (s.h_bound[b] < 0 ? BP_ERANGE : BP_OK);
        res.latency_us =
            std::chrono::duration<double, std::micro>(now - r.t_submit).count();
        S->completed.push_back(res);
        S->queued_items -= (int64_t)r.assign.size();
        S->n_done++;
      }
      if (err) S->worker_status = BP_ECUDA;
      s.batch.clear();
      s.busy = false;
      s.failed = false;
      did = true;
      S->cv_done.notify_all();
    }
    // 2. new batches
    for (Slot &s : S->slots) {
      if (s.busy) continue;
      int32_t n_inst;
      {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->pending.empty()) break;
        int64_t items = 0;
        while (!S->pending.empty() && (int32_t)s.batch.size() < S->max_batch) {
          const int64_t n = (int64_t)S->pending.front().assign.size();
          if (!s.batch.empty() && items + n > S->slot_items) break;
          items += n;
          s.batch.push_back(std::move(S->pending.front()));
          S->pending.pop_front();
        }
        n_inst = S->n_instances;
        S->n_batches++;
      }
      s.busy = true;
      s.failed = launch_slot(S, s, n_inst) != BP_OK;  // reported at the next collection
      did = true;
    }
    if (S->stop.load()) {
      bool idle = true;
      for (Slot &s : S->slots) idle &= !s.busy;
      std::lock_guard<std::mutex> lock(S->mu);
      if (idle && S->pending.empty()) break;
    }
    if (!did) {
      std::unique_lock<std::mutex> lock(S->mu);
      bool any_busy = false;
      for (Slot &s : S->slots) any_busy |= s.busy;
      // poll in-flight batches every 20 us; sleep up to 2 ms when idle
      S->cv_work.wait_for(lock, std::chrono::microseconds(any_busy ? 20 : 2000));
    }
  }
}

}  // namespace

extern "C" {

int bp_serve_create(int64_t pool_items, int32_t max_instances, int64_t max_queued_items,
                    int32_t slots, int32_t max_batch, int64_t max_bins, bp_serve_t **out) {
  if (!out) return BP_EINVAL;
  *out = nullptr;
  if (pool_items < 1 || max_instances < 1 || max_queued_items < 1 || slots < 1 || slots > 16 ||
      max_batch < 1 || max_bins < 0 || max_bins > 16384)
    return BP_ERANGE;
  bp_serve *S = new (std::nothrow) bp_serve();
  if (!S) return BP_ENOMEM;
  S->pool_items = pool_items;
  S->max_instances = max_instances;
  S->max_queued_items = max_queued_items;
  S->max_batch = max_batch;
  S->max_bins = max_bins;
  // each slot stages up to max_queued_items / slots assignment entries; no
  // single registered instance may be larger
  S->slot_items = std::max<int64_t>(1, max_queued_items / slots);
  int st = cuda_st(cudaGetDevice(&S->device));
  if (st == BP_OK) st = cuda_st(cudaMalloc(&S->d_pool, sizeof(int32_t) * (size_t)pool_items));
  if (st == BP_OK)
    st = cuda_st(cudaMalloc(&S->d_pool_off, sizeof(int64_t) * ((size_t)max_instances + 1)));
  if (st == BP_OK) st = cuda_st(cudaMalloc(&S->d_pool_cap, sizeof(int64_t) * (size_t)max_instances));
  if (st == BP_OK) st = cuda_st(cudaMemset(S->d_pool_off, 0, sizeof(int64_t)));
  S->pool_off.assign(1, 0);
  S->slots.resize(slots);
  for (int i = 0; i < slots && st == BP_OK; ++i) {
    st = alloc_slot(S->slots[i], S->slot_items, max_batch);
  }
  if (st != BP_OK) {
    for (Slot &s : S->slots) free_slot(s);
    cudaFree(S->d_pool);
    cudaFree(S->d_pool_off);
    cudaFree(S->d_pool_cap);
    delete S;
    return st;
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return BP_OK;
}

int bp_serve_destroy(bp_serve_t *S) {
  if (!S) return BP_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop.store(true);
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaDeviceSynchronize();
  for (Slot &s : S->slots) free_slot(s);
  cudaFree(S->d_pool);
  cudaFree(S->d_pool_off);
  cudaFree(S->d_pool_cap);
  delete S;
  return BP_OK;
}

int bp_serve_register(bp_serve_t *S, const int32_t *sizes, int64_t n, int64_t capacity,
                      int32_t *out_id) {
  if (!S || !out_id || n < 0 || (n > 0 && !sizes)) return BP_EINVAL;
  if (capacity < 1 || capacity > (int64_t(1) << 30) || n > S->slot_items) return BP_ERANGE;
  for (int64_t i = 0; i < n; ++i)
    if (sizes[i] < 0 || (int64_t)sizes[i] > capacity) return BP_ERANGE;
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->n_instances >= S->max_instances || S->pool_off.back() + n > S->pool_items) {
    S->n_refused++;
    return BP_EBUSY;
  }
  const int32_t id = S->n_instances;
  const int64_t off = S->pool_off.back();
  int st = BP_OK;
  // synchronous copies: the new entries are not yet visible to any batch
  if (n > 0)
    st = cuda_st(cudaMemcpy(S->d_pool + off, sizes, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  const int64_t end = off + n;
  if (st == BP_OK)
    st = cuda_st(cudaMemcpy(S->d_pool_off + id + 1, &end, sizeof(int64_t), cudaMemcpyHostToDevice));
  if (st == BP_OK)
    st = cuda_st(cudaMemcpy(S->d_pool_cap + id, &capacity, sizeof(int64_t), cudaMemcpyHostToDevice));
  if (st != BP_OK) return st;
  S->pool_off.push_back(end);
  S->pool_cap.push_back(capacity);
  S->n_instances = id + 1;
  *out_id = id;
  return BP_OK;
}

int bp_serve_submit(bp_serve_t *S, int32_t instance, const int32_t *assign, int64_t bins,
                    int64_t tag, int64_t *out_request) {
  if (!S || instance < 0) return BP_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (instance >= S->n_instances) return BP_EINVAL;
  if (bins < 0 || bins > S->max_bins) return BP_ERANGE;
  const int64_t n = S->pool_off[instance + 1] - S->pool_off[instance];
  if (n > 0 && !assign) return BP_EINVAL;
  if (S->worker_status != BP_OK) return S->worker_status;
  if (S->queued_items + n > S->max_queued_items && S->queued_items > 0) {
    S->n_refused++;
    return BP_EBUSY;
  }
  Request r;
  r.id = S->next_id++;
  r.tag = tag;
  r.instance = instance;
  r.bins = bins;
  r.assign.assign(assign, assign + n);
  r.t_submit = Clock::now();
  S->queued_items += n;
  if (out_request) *out_request = r.id;
  S->pending.push_back(std::move(r));
  S->cv_work.notify_one();
  return BP_OK;
}

int bp_serve_poll(bp_serve_t *S, bp_serve_result_t *out, int32_t max_results, int32_t *count,
                  int32_t wait_us) {
  if (!S || !count || max_results < 0 || (max_results > 0 && !out)) return BP_EINVAL;
  std::unique_lock<std::mutex> lock(S->mu);
  if (S->completed.empty() && wait_us > 0)
    S->cv_done.wait_for(lock, std::chrono::microseconds(wait_us),
                        [S] { return !S->completed.empty(); });
  const int32_t k = (int32_t)std::min<size_t>((size_t)max_results, S->completed.size());
  std::copy(S->completed.begin(), S->completed.begin() + k, out);
  S->completed.erase(S->completed.begin(), S->completed.begin() + k);
  *count = k;
  if (k == 0 && wait_us > 0) return BP_ETIMEOUT;
  return BP_OK;
}

int bp_serve_stats(bp_serve_t *S, int64_t *pending, int64_t *queued_items, int64_t *batches,
                   int64_t *done, int64_t *refused) {
  if (!S) return BP_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (pending) *pending = (int64_t)S->pending.size();
  if (queued_items) *queued_items = S->queued_items;
  if (batches) *batches = S->n_batches;
  if (done) *done = S->n_done;
  if (refused) *refused = S->n_refused;
  return S->worker_status;
}

}  // extern "C"
