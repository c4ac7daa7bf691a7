// Request server: continuous batching of least-squares solves on one GPU.
//
// snsolve_server_create allocates, once, a device workspace arena (all solver
// scratch of admitted requests is carved from it; nothing is allocated while
// serving) and starts one worker thread per slot, each with its own CUDA stream.
// snsolve_submit queues a request.  A request's footprint is the bytes of its
// resident inputs (A and b, owned by the caller) plus its solver workspace.
// A free slot takes the oldest pending request that fits (the sum of the
// admitted footprints stays within the HBM budget and the arena has room), so a
// large request that must wait for memory does not block smaller ones behind
// it; the oldest request can be passed over at most 2 x slots times, after
// which nothing overtakes it until it is admitted (no starvation).  A request
// whose footprint alone exceeds the budget is refused (SNS_EBUDGET).
// Admitted requests run concurrently on their slots' streams, so their kernels
// overlap on the device, and a newly arrived request starts as soon as a slot
// and memory free up, without waiting for the others (continuous batching).
// snsolve_poll waits, bounded, for a request's completion.
#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "snsolve.h"
#include "fault.h"

namespace sns {
sns_status record_cuda_error(cudaError_t e);
}

namespace {

// First-fit allocator over [0, size) with coalescing, 256-byte granularity.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (!bytes) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rem = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rem) free_[noff] = rem;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (!bytes) bytes = 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0;
};

struct Req {
  uint64_t id;
  sns_problem prob;
  sns_opts opts;
  double* x;
  size_t ws_bytes, footprint;
  int bypassed = 0;     // times a younger request was admitted ahead of this one
};
struct Result {
  bool done = false;
  sns_info info{};
};

}  // namespace

struct sns_server {
  sns_ctx* ctx = nullptr;
  size_t budget = 0, used = 0;
  int max_slots = 0, running = 0;
  uint8_t* arena_base = nullptr;
  Arena arena;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req> pending;
  std::unordered_map<uint64_t, Result> results;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  uint64_t next_id = 1;
  bool stop = false;
  int device = 0;
};

static size_t input_bytes(const sns_problem* p) {
  switch (p->fmt) {
    case SNS_DENSE_F32: return (size_t)p->m * p->lda * 4 + (size_t)p->m * 4;
    case SNS_DENSE_F64: return (size_t)p->m * p->lda * 8 + (size_t)p->m * 8;
    case SNS_CSR_F32: return (size_t)(p->m + 1) * 8 + (size_t)p->nnz * 8 + (size_t)p->m * 4;
  }
  return 0;
}

static void worker_loop(sns_server* S, int slot) {
  cudaSetDevice(S->device);
  cudaStream_t st = S->streams[slot];
  for (;;) {
    Req r;
    size_t off = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) return;
        // first fit in arrival order, the oldest request passed over a bounded number of times
        bool took = false;
        const int bypass_limit = 2 * S->max_slots;
        for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
          if (it != S->pending.begin() && S->pending.front().bypassed >= bypass_limit) break;
          if (S->used + it->footprint <= S->budget && S->arena.alloc(it->ws_bytes, &off)) {
            r = *it;
            if (it != S->pending.begin()) S->pending.front().bypassed++;
            S->pending.erase(it);
            S->used += r.footprint;
            S->running++;
            took = true;
            break;
          }
        }
        if (took) break;
        S->cv_work.wait(lk);
      }
    }
    sns_info info{};
    sns_status s = snsolve_lstsq(S->ctx, &r.prob, &r.opts, r.x, &info, S->arena_base + off, r.ws_bytes, st);
    if (s != SNS_OK && info.status == SNS_OK) info.status = s;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->arena.release(off, r.ws_bytes);
      S->used -= r.footprint;
      S->running--;
      Result& res = S->results[r.id];
      res.done = true;
      res.info = info;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

extern "C" {

sns_status snsolve_server_create(sns_server** out, sns_ctx* ctx, size_t hbm_budget_bytes, int max_slots) {
  if (!out) return SNS_EINVAL;
  *out = nullptr;
  if (!ctx || hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 256) return SNS_EINVAL;
  sns_server* S = new sns_server();
  S->ctx = ctx;
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  cudaGetDevice(&S->device);
  // arena for solver scratch: a quarter of the budget, at most 32 GiB
  size_t arena = hbm_budget_bytes / 4;
  const size_t cap = (size_t)32 << 30;
  if (arena > cap) arena = cap;
  arena = (arena + 255) & ~(size_t)255;
  if (sns::fault_hit(sns::kFaultAlloc)) {
    delete S;
    return sns::record_injected("injected allocation failure", SNS_ENOMEM);
  }
  cudaError_t e = cudaMalloc(&S->arena_base, arena);
  if (e != cudaSuccess) {
    delete S;
    sns::record_cuda_error(e);
    return SNS_ENOMEM;
  }
  S->arena.init(arena);
  S->streams.resize(max_slots);
  for (int i = 0; i < max_slots; ++i) {
    e = cudaStreamCreateWithFlags(&S->streams[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaStreamDestroy(S->streams[j]);
      cudaFree(S->arena_base);
      delete S;
      return sns::record_cuda_error(e);
    }
  }
  for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker_loop, S, i);
  *out = S;
  return SNS_OK;
}

void snsolve_server_destroy(sns_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto st : S->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(S->arena_base);
  delete S;
}

sns_status snsolve_submit(sns_server* S, const sns_problem* prob, const sns_opts* opts, double* x,
                          uint64_t* req_id) {
  if (!S || !prob || !opts || !x || !req_id) return SNS_EINVAL;
  size_t ws = 0;
  sns_status s = snsolve_lstsq_workspace_size(prob, opts, &ws);
  if (s != SNS_OK) return s;
  Req r;
  r.prob = *prob;
  r.opts = *opts;
  r.x = x;
  r.ws_bytes = (ws + 255) & ~(size_t)255;
  r.footprint = input_bytes(prob) + r.ws_bytes;
  if (r.footprint > S->budget || r.ws_bytes > S->arena.size()) return SNS_EBUDGET;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r.id = S->next_id++;
    S->results[r.id];   // pending entry
    S->pending.push_back(r);
    *req_id = r.id;
  }
  S->cv_work.notify_one();
  return SNS_OK;
}

sns_status snsolve_poll(sns_server* S, uint64_t req_id, int64_t timeout_us, sns_info* info) {
  if (!S) return SNS_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->results.find(req_id);
  if (it == S->results.end()) return SNS_EINVAL;
  if (!it->second.done && timeout_us > 0) {
    S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] {
      auto jt = S->results.find(req_id);
      return jt != S->results.end() && jt->second.done;
    });
    it = S->results.find(req_id);
  }
  if (!it->second.done) return timeout_us > 0 ? SNS_ETIMEOUT : SNS_EAGAIN;
  if (info) *info = it->second.info;
  S->results.erase(it);
  return SNS_OK;
}

sns_status snsolve_server_stats(sns_server* S, int* running, int* pending, size_t* used_bytes) {
  if (!S) return SNS_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (running) *running = S->running;
  if (pending) *pending = (int)S->pending.size();
  if (used_bytes) *used_bytes = S->used;
  return SNS_OK;
}

}  // extern "C"
