// Per-kernel timing and launch counting (see prof.h).  Timing is off unless
// snsolve_profile(1) is called; the launch counter always runs.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "prof.h"
#include "snsolve_debug.h"

namespace sns {

static const char* kNames[K_COUNT] = {
    "cs_sort_blocks", "cs_gather_dense", "cs_stream_dense", "cs_gather_csr", "srht_sample", "srht_pass1",
    "srht_pass2",     "gauss_apply",     "qr_load",         "qr_house",      "rinv",        "resid_pass",
    "normal_pass",    "pcg_matvec",      "pcg_apply",       "eta",           "batched",     "misc",
    "saa_form_y",     "cs_apply"};

const char* kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? kNames[id] : "?"; }

static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_on{0};

struct Rec {
  int id;
  cudaEvent_t a, b;
};
static std::mutex g_mu;
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static thread_local int t_span_depth = 0;

ProfScope::ProfScope(int id, cudaStream_t st) : id_(id), st_(st), slot_(-1) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_on.load(std::memory_order_relaxed) && t_span_depth == 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{id, get_event(), get_event()};
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    slot_ = (int)g_recs.size() - 1;
  }
}

ProfScope::~ProfScope() {
  if (slot_ >= 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot_ < (int)g_recs.size()) cudaEventRecord(g_recs[slot_].b, st_);
  }
}

ProfSpan::ProfSpan(int id, cudaStream_t st) : st_(st), slot_(-1) {
  if (g_on.load(std::memory_order_relaxed) && t_span_depth == 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    Rec r{id, get_event(), get_event()};
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    slot_ = (int)g_recs.size() - 1;
  }
  ++t_span_depth;
}

ProfSpan::~ProfSpan() {
  --t_span_depth;
  if (slot_ >= 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot_ < (int)g_recs.size()) cudaEventRecord(g_recs[slot_].b, st_);
  }
}

}  // namespace sns

using namespace sns;

extern "C" {

uint64_t snsolve_launch_count(void) { return g_launches.load(); }

int snsolve_profile_num_kernels(void) { return K_COUNT; }

const char* snsolve_profile_kernel_name(int id) { return kernel_name(id); }

sns_status snsolve_profile(int enable) {
  g_on.store(enable ? 1 : 0);
  return SNS_OK;
}

sns_status snsolve_profile_read(double* ms, uint64_t* count, int nid) {
  if (!ms || !count || nid < K_COUNT) return SNS_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < nid; ++i) { ms[i] = 0.0; count[i] = 0; }
  for (auto& r : g_recs) {
    cudaEventSynchronize(r.b);
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.id] += t;
      count[r.id] += 1;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  return SNS_OK;
}

}  // extern "C"
