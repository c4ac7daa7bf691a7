// Shared device helpers of the snsolve CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "snsolve.h"
#include "fault.h"

#define SNS_HD __host__ __device__ __forceinline__
#define SNS_D __device__ __forceinline__

namespace sns {

// ---------------------------------------------------------------------------
// Counter-based random stream defining the implicit sketch (generate-S step,
// Sec. 1.2): SplitMix64 of Steele, Lea & Flood (OOPSLA 2014).  Output i of a
// generator whose state starts at s0 is mix64(s0 + (i + 1) * gamma).
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMul1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMul2 = 0x94D049BB133111EBull;

enum Stream : uint64_t {
  kStreamCountSketch = 0,
  kStreamSrhtSign = 1,
  kStreamSrhtSample = 2,
  kStreamGaussian = 3,
  kStreamSparseSign = 4      // draws 1.. of the sparse sign embedding
};

SNS_HD uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * kMul1;
  z = (z ^ (z >> 27)) * kMul2;
  return z ^ (z >> 31);
}
SNS_HD uint64_t stream_state(uint64_t seed, uint64_t stream) { return seed ^ (stream << 56); }
SNS_HD uint64_t splitmix_at(uint64_t s0, uint64_t idx) { return mix64(s0 + (idx + 1) * kGamma); }
// State whose output i is output i + offset of the stream that starts at s0:
// splitmix_at(shift_state(s0, o), i) == splitmix_at(s0, i + o).  A sketch of
// rows row0.. of a larger matrix uses it so every row keeps its global index.
SNS_HD uint64_t shift_state(uint64_t s0, uint64_t offset) { return s0 + offset * kGamma; }

// Multiply-shift range reduction of the low 32 bits into [0, d) (Lemire 2019).
SNS_HD uint32_t bucket_of(uint64_t key, uint64_t d) {
  return (uint32_t)(((key & 0xFFFFFFFFull) * d) >> 32);
}
// Sign: bit 63 set -> -1.
SNS_HD float sign_of(uint64_t key) { return (key >> 63) ? -1.0f : 1.0f; }

// ---------------------------------------------------------------------------
SNS_D float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
SNS_D double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
SNS_D double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of doubles; every thread gets the result.  `red` holds >= 32
// doubles of shared memory.  Must be called by all threads of the block.
SNS_D double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];   // fixed order: deterministic
  return t;
}

// ---------------------------------------------------------------------------
// Error-free transformations for FP64-class accumulation on the FP32 pipes
// (Dekker 1971; Knuth TAOCP vol. 2, 4.2.2): a float-float value is hi + lo with
// |lo| <= ulp(hi)/2.
struct ff {
  float hi, lo;
};
SNS_D ff two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
SNS_D ff fast_two_sum(float a, float b) {  // requires |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
// (hi, lo) += a * b exactly for the product (TwoProdFMA) and to float-float
// accuracy for the sum.
SNS_D void ff_fma(ff& acc, float a, float b) {
  float p = a * b;
  float pe = fmaf(a, b, -p);
  ff s = two_sum(acc.hi, p);
  s.lo += acc.lo + pe;
  acc = fast_two_sum(s.hi, s.lo);
}
SNS_D void ff_add(ff& acc, ff v) {
  ff s = two_sum(acc.hi, v.hi);
  s.lo += acc.lo + v.lo;
  acc = fast_two_sum(s.hi, s.lo);
}
SNS_D ff ff_from_double(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}
SNS_D double ff_to_double(ff v) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------------------------
// Bounded spin on a device flag: returns true once *flag >= target, false
// after `limit` polls (the caller records an error and leaves).
SNS_D bool spin_until_ge(const volatile int* flag, int target, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    if (*flag >= target) return true;
    if (it >= 4096) __nanosleep(32);   // tight polling first: the flags of the QR flip within microseconds
  }
  return *flag >= target;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// launch_dependent() may become resident while the previous kernel of the
// stream is still finishing; it must call grid_dep_wait() before it reads
// anything that kernel wrote (work on read-only inputs may come first).
// grid_dep_trigger() lets the next dependent kernel start launching; a CTA
// that exits triggers implicitly.  Without the launch attribute both are no-ops.
SNS_D void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
SNS_D void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
SNS_D void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

}  // namespace sns

// Host-side launch error check used by the dispatch layer.
#define SNS_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return sns::record_cuda_error(_e); \
  } while (0)

// After a kernel launch: the launch's own error, or a host-side injected
// launch failure (fault.h).
#define SNS_LAUNCH_CHECK()                                                        \
  do {                                                                            \
    if (::sns::fault_hit(::sns::kFaultLaunch))                                    \
      return ::sns::record_injected("injected launch failure", SNS_ECUDA);       \
    SNS_CUDA_TRY(cudaGetLastError());                                             \
  } while (0)

namespace sns {
sns_status record_cuda_error(cudaError_t e);
// Raises a kernel's dynamic shared-memory limit to the device maximum, once per
// (device, kernel).  Kernels are launched with varying dynamic sizes from
// several host threads; setting the limit per call would let one thread lower
// it between another thread's set and launch.
cudaError_t raise_smem_limit(const void* func);

// Launches kernel<<<grid, block, smem, st>>>(args...) as a programmatic
// dependent of the stream's previous kernel (see grid_dep_wait).
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
}
