// Optional per-kernel timing (CUDA events recorded on the launch stream around
// each launch) and a global launch counter.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sns {

enum KernelId {
  K_CS_SORT = 0, K_CS_GATHER, K_CS_STREAM, K_CS_CSR, K_SRHT_SAMPLE, K_SRHT_PASS1, K_SRHT_PASS2, K_GAUSS,
  K_QR_LOAD, K_QR, K_RINV, K_RESID, K_NORMAL, K_MATVEC, K_CG, K_ETA, K_BATCH, K_MISC, K_SAA_Y, K_CS_APPLY, K_COUNT
};
const char* kernel_name(int id);

// RAII scope around one launch: counts it and, when profiling is on, records
// a start/stop event pair on `st`.
class ProfScope {
 public:
  ProfScope(int id, cudaStream_t st);
  ~ProfScope();

 private:
  int id_;
  cudaStream_t st_;
  int slot_;
};

// RAII scope around several launches that must stay adjacent on the stream (a
// kernel and its programmatic dependent): one start/stop event pair for the
// whole span when profiling is on; the launches inside it are counted but get
// no events of their own (an event between them would serialise the pair).
class ProfSpan {
 public:
  ProfSpan(int id, cudaStream_t st);
  ~ProfSpan();

 private:
  cudaStream_t st_;
  int slot_;
};

}  // namespace sns

#define SNS_PROF(id, st) ::sns::ProfScope _sns_prof_scope_(id, st)
