// CountSketch apply for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) when they want a
// sketch: code running inside a host callback or another library's critical
// section, allocators that must not grow after start-up, or processes whose
// device memory is fully reserved up front.  snsolve_sketch needs a
// caller-provided workspace; this entry point instead uses a fixed scratch
// array that is part of the library's device image.  Every GPU that loads the
// library holds this array (kStaticScratchBytes) until the process exits.
//
// It runs the same bucket-sorted (deterministic) CountSketch kernels as
// snsolve_sketch with variant SNS_CS_SORTED, on dense FP32 input only, and
// always with the two-kernel plan and the warp gather: neither waits on the
// device, so a call cannot time out there and leaves no status word behind
// (the cooperative plan and the bulk-copy gather, which do wait, are never
// selected here; the results are the same).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "snsolve.h"

namespace sns {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;   // 16 MiB

// The scratch.  Host code must not pass &g_static_scratch to a kernel: on the
// host that name is only a stand-in for the device symbol.  The device address
// comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void* g_static_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device with that device current.
static sns_status static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return record_cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices) return SNS_EINVAL;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return record_cuda_error(e);
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SNS_OK;
}

}  // namespace sns

using namespace sns;

extern "C" {

sns_status snsolve_sketch_countsketch_static(const sns_problem* prob, int64_t d, uint64_t seed, float* SA,
                                             int64_t ldsa, float* Sb, void* stream) {
  if (!prob || !SA || !Sb || !prob->A || !prob->b) return SNS_EINVAL;
  if (prob->fmt != SNS_DENSE_F32) return SNS_EINVAL;
  if (prob->m < 1 || prob->n < 1 || prob->m < prob->n || prob->lda < prob->n || prob->m >= ((int64_t)1 << 31))
    return SNS_EINVAL;
  if (d < prob->n || d < 1 || d > cs_sorted_max_d() || ldsa < prob->n) return SNS_EINVAL;
  const CsLayout L = cs_layout(prob->m, prob->n, d, false, false);
  if (L.bytes > kStaticScratchBytes) return SNS_ENOMEM;    // problem too large for the fixed scratch
  void* scratch = nullptr;
  sns_status s = static_scratch(&scratch);
  if (s != SNS_OK) return s;
  // The kernels write every scratch byte they later read (phase 1 writes the
  // row order and segment table and clears the bucket counters), so leftovers
  // from an earlier call need no clearing here.
  DenseArgs a{prob->A, prob->lda, prob->b, prob->m, prob->n, false};
  return cs_apply_dense_sorted(a, d, seed, SA, ldsa, Sb, 1, scratch, kStaticScratchBytes,
                               static_cast<cudaStream_t>(stream), /*allow_bulk=*/false);
}

}  // extern "C"
