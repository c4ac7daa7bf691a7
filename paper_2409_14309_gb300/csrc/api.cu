// C ABI of snsolve: argument validation, workspace layout and the solve driver
// (sketch -> FP64 QR -> back-solve -> optional preconditioned refinement).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <mutex>
#include <set>

#include "common.cuh"
#include "kernels.h"
#include "snsolve.h"
#include "snsolve_debug.h"

struct sns_ctx {
  int device;
  double* pinned;   // host pinned scalars (eta, ||r||, ||g||, ||A||_F, status, sres, ...)
};

namespace sns {

static thread_local char t_err[256] = "";

sns_status record_cuda_error(cudaError_t e) {
  snprintf(t_err, sizeof(t_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return SNS_ECUDA;
}
sns_status record_injected(const char* what, sns_status s) {
  snprintf(t_err, sizeof(t_err), "%s", what);
  return s;
}

static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// Stopping tolerances at or above this use the cheaper g = A^T r accumulation
// of the residual pass (FP32 products, compensated sums): its eta floor is at
// most ~3e-8, so eta is still resolved to a few percent at 1e-6.
constexpr double kCheapGradTol = 1e-6;
// Upper bound on inner CG steps per refinement cycle when the caller sets none;
// cycles normally end earlier, on the device.
constexpr int kDefaultInnerMax = 8;
// The preconditioner M^-1 = R^-1 R^-T is applied as one formed matrix P while
// max|R_ii| / min|R_ii| (a lower bound on kappa(R), measured 20-30x below it on
// Gaussian-based test matrices) stays below this; above it, as two triangular
// products, since P's FP64 rounding (relative to kappa(R)^2) would leave it
// indefinite.
constexpr double kFactoredDiagRatio = 5e5;

cudaError_t raise_smem_limit(const void* func) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, func})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes attr;
  e = cudaFuncGetAttributes(&attr, func);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)attr.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({dev, func});
  return e;
}

// Pinned host scalars for the convergence checks of snsolve_lstsq, one block
// per host thread, so concurrent calls on one context do not share them.
struct PinnedScalars {
  double* p = nullptr;
  ~PinnedScalars() {
    if (p) cudaFreeHost(p);
  }
};
static thread_local PinnedScalars t_pinned;

// Per-thread side stream and events (created once per host thread).
struct SideStream {
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool ok = false;
  int device = -1;
  ~SideStream() {
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (st) cudaStreamDestroy(st);
  }
};
static thread_local SideStream t_side;
static SideStream& thread_side_stream() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (!t_side.ok || t_side.device != dev) {
    t_side.ok = cudaStreamCreateWithFlags(&t_side.st, cudaStreamNonBlocking) == cudaSuccess &&
                cudaEventCreateWithFlags(&t_side.ev_in, cudaEventDisableTiming) == cudaSuccess &&
                cudaEventCreateWithFlags(&t_side.ev_out, cudaEventDisableTiming) == cudaSuccess;
    t_side.device = dev;
  }
  return t_side;
}
static double* thread_pinned() {
  if (!t_pinned.p) {
    if (fault_hit(kFaultAlloc)) {
      record_injected("injected allocation failure", SNS_ENOMEM);
      return nullptr;
    }
    if (cudaHostAlloc(&t_pinned.p, 4096, cudaHostAllocDefault) != cudaSuccess) t_pinned.p = nullptr;
  }
  return t_pinned.p;
}

static bool is_f64(const sns_problem* p) { return p->fmt == SNS_DENSE_F64; }

static sns_status validate_problem(const sns_problem* p) {
  if (!p) return SNS_EINVAL;
  if (p->m < 1 || p->n < 1 || p->m < p->n || p->m >= ((int64_t)1 << 31)) return SNS_EINVAL;
  if (!p->b) return SNS_EINVAL;
  if (p->fmt == SNS_DENSE_F32 || p->fmt == SNS_DENSE_F64) {
    if (!p->A || p->lda < p->n) return SNS_EINVAL;
  } else if (p->fmt == SNS_CSR_F32) {
    if (!p->rowptr || (p->nnz > 0 && (!p->col || !p->val)) || p->nnz < 0) return SNS_EINVAL;
  } else {
    return SNS_EINVAL;
  }
  return SNS_OK;
}

static int64_t next_pow2(int64_t m) {
  int64_t p = 1;
  while (p < m) p <<= 1;
  return p;
}

static sns_status validate_sketch(const sns_problem* p, const sns_sketch_desc* sk) {
  if (!sk) return SNS_EINVAL;
  if (sk->d < p->n || sk->d < 1 || sk->d > ((int64_t)1 << 24)) return SNS_EINVAL;
  switch (sk->kind) {
    case SNS_COUNTSKETCH:
      if (sk->variant < SNS_CS_AUTO || sk->variant > SNS_CS_STREAM) return SNS_EINVAL;
      if (sk->variant == SNS_CS_SORTED && sk->d > cs_sorted_max_d()) return SNS_EINVAL;
      if (sk->variant == SNS_CS_STREAM && p->fmt == SNS_DENSE_F64) return SNS_EINVAL;
      if (p->fmt == SNS_CSR_F32 && sk->variant == SNS_CS_SORTED && sk->d > cs_sorted_max_d()) return SNS_EINVAL;
      if (p->fmt == SNS_CSR_F32 && sk->variant == SNS_CS_SORTED && p->n > cs_csr_sorted_max_n()) return SNS_EINVAL;
      if (p->fmt == SNS_CSR_F32 && p->n > 50000) return SNS_EINVAL;
      return SNS_OK;
    case SNS_GAUSSIAN:
      if (p->fmt != SNS_DENSE_F32) return SNS_EINVAL;
      if (sk->variant < 0 || sk->variant > 3) return SNS_EINVAL;   // BF16 terms of A (0: auto)
      return SNS_OK;
    case SNS_SRHT:
      if (p->fmt == SNS_CSR_F32) return SNS_EINVAL;
      if (sk->d > next_pow2(p->m) || next_pow2(p->m) >= ((int64_t)1 << 31)) return SNS_EINVAL;
      return SNS_OK;
    case SNS_SPARSE_SIGN:
      if (p->fmt != SNS_DENSE_F32) return SNS_EINVAL;
      if (sk->variant < 1 || sk->variant > 8 || sk->variant > sk->d) return SNS_EINVAL;
      return SNS_OK;
    default:
      return SNS_EINVAL;
  }
}

// CountSketch variant: FP64 dense is always sorted; CSR is sorted only when
// asked for (the sorted CSR sketch and the deterministic CSR passes it selects
// cost ~2.5x the streaming ones, measured); FP32 dense is sorted unless asked
// otherwise or d is above the sorted variant's limit.
static bool cs_use_sorted(const sns_problem* p, const sns_sketch_desc* sk) {
  if (p->fmt == SNS_DENSE_F64) return true;
  if (sk->variant == SNS_CS_STREAM) return false;
  if (sk->variant == SNS_CS_SORTED) return true;
  if (p->fmt == SNS_CSR_F32) return false;
  return sk->d <= cs_sorted_max_d();
}

// BF16 terms of A in the tensor-core Gaussian product; AUTO is one term for a
// sketch returned to the caller (solve paths resolve it first: solve_sketch).
static int gauss_terms(const sns_sketch_desc* sk) { return sk->variant == 0 ? 1 : sk->variant; }

// The sketch a solve applies: AUTO Gaussian becomes three BF16 terms (FP32 A
// exactly), since R of a one-term sketch preconditions an ill-conditioned A
// poorly (kappa(A R^-1) grows with kappa(A) * 2^-9).
static sns_sketch_desc solve_sketch(const sns_opts* o) {
  sns_sketch_desc sk = o->sk;
  if (sk.kind == SNS_GAUSSIAN && sk.variant == 0) sk.variant = 3;
  return sk;
}

static size_t sketch_ws(const sns_problem* p, const sns_sketch_desc* sk) {
  switch (sk->kind) {
    case SNS_COUNTSKETCH:
      if (!cs_use_sorted(p, sk)) return 0;
      return cs_layout(p->m, p->n, sk->d, is_f64(p), p->fmt == SNS_CSR_F32).bytes;
    case SNS_GAUSSIAN:
      return gauss_ws_bytes(p->m, p->n, sk->d, gauss_terms(sk));
    case SNS_SRHT:
      return srht_ws_bytes(p->m, p->n, sk->d, is_f64(p));
    case SNS_SPARSE_SIGN:
      return 0;
  }
  return 0;
}

// Error word of the sketch kernels that wait on the device with bounded waits
// (the tcgen05 Gaussian kernel, the bulk-copy CountSketch gather), or null.
static const void* sketch_err_word(const sns_problem* p, const sns_sketch_desc* sk, const uint8_t* skws) {
  if (sk->kind == SNS_GAUSSIAN) return skws + gauss_err_offset();
  if (sk->kind == SNS_COUNTSKETCH && p->fmt == SNS_DENSE_F32 && cs_use_sorted(p, sk))
    return skws + cs_layout(p->m, p->n, sk->d, false, false).off_err;
  return nullptr;
}

static sns_status run_sketch(const sns_problem* p, const sns_sketch_desc* sk, void* SA, int64_t ldsa, void* Sb,
                             int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st, int64_t row0 = 0) {
  DenseArgs da{p->A, p->lda, p->b, p->m, p->n, is_f64(p), row0};
  switch (sk->kind) {
    case SNS_COUNTSKETCH:
      if (p->fmt == SNS_CSR_F32) {
        CsrArgs ca{p->rowptr, p->col, p->val, static_cast<const float*>(p->b), p->m, p->n, p->nnz, row0};
        if (!cs_use_sorted(p, sk))
          return cs_apply_csr_stream(ca, sk->d, sk->seed, static_cast<float*>(SA), ldsa, static_cast<float*>(Sb),
                                     sbs, st);
        return cs_apply_csr(ca, sk->d, sk->seed, static_cast<float*>(SA), ldsa, static_cast<float*>(Sb), sbs, ws,
                            ws_bytes, st);
      }
      if (cs_use_sorted(p, sk)) return cs_apply_dense_sorted(da, sk->d, sk->seed, SA, ldsa, Sb, sbs, ws, ws_bytes, st);
      return cs_apply_dense_stream(da, sk->d, sk->seed, SA, ldsa, Sb, sbs, st);
    case SNS_GAUSSIAN:
      return gauss_apply_dense(da, sk->d, sk->seed, gauss_terms(sk), static_cast<float*>(SA), ldsa,
                               static_cast<float*>(Sb), sbs, ws,
                               ws_bytes, st);
    case SNS_SRHT:
      return srht_apply_dense(da, sk->d, sk->seed, SA, ldsa, Sb, sbs, ws, ws_bytes, st);
    case SNS_SPARSE_SIGN:
      return cs_apply_sparse_sign(da, sk->d, sk->variant, sk->seed, static_cast<float*>(SA), ldsa,
                                  static_cast<float*>(Sb), sbs, st);
  }
  return SNS_EINVAL;
}

// Workspace of snsolve_lstsq.
struct LsLayout {
  size_t off_saug, off_sk, sk_bytes, off_w, off_dev, off_qr, off_iter, off_y, bytes;
  int grid;
};
static bool uses_saa(const sns_opts* o) { return o->tol > 0 && o->method == SNS_SAA; }
static LsLayout ls_layout(const sns_problem* p, const sns_opts* o) {
  LsLayout L{};
  const int64_t d = o->sk.d, q = p->n + 1;
  const size_t esz = is_f64(p) ? 8 : 4;
  size_t off = 0;
  L.off_saug = off; off += al((size_t)d * q * esz);
  const sns_sketch_desc sk = solve_sketch(o);
  L.sk_bytes = sketch_ws(p, &sk);
  L.off_sk = off; off += al(L.sk_bytes);
  L.off_w = off; off += al((size_t)d * q * 8);
  L.off_dev = off; off += al(64);
  L.off_qr = off; off += al(qr_coop_ws_bytes(d, q));
  L.grid = iter_grid();
  L.off_iter = off;
  if (o->tol > 0) off += al(iter_ws_bytes(p->n, L.grid));
  L.off_y = off;
  if (uses_saa(o)) off += al(saa_y_bytes(p->m, p->n, is_f64(p)));
  L.bytes = off;
  return L;
}

static sns_status validate_opts(const sns_problem* p, const sns_opts* o) {
  if (!o) return SNS_EINVAL;
  sns_status s = validate_sketch(p, &o->sk);
  if (s != SNS_OK) return s;
  if (o->max_iter < 0 || o->inner < 0) return SNS_EINVAL;
  if (p->fmt == SNS_CSR_F32 && o->sk.kind == SNS_COUNTSKETCH && o->sk.variant == SNS_CS_SORTED &&
      p->n > csr_det_max_n())
    return SNS_EINVAL;   // reproducible passes keep per-warp rows of n doubles in shared memory
  if (o->sk.d > 16384) return SNS_EINVAL;   // the QR keeps one column of SA in shared memory
  if (o->tol > 0 && p->fmt != SNS_CSR_F32 && p->n > 1024) return SNS_EINVAL;
  if (!(o->tol == o->tol)) return SNS_EINVAL;  // NaN
  if (o->method != SNS_SAP && o->method != SNS_SAA) return SNS_EINVAL;
  if (o->method == SNS_SAA && (p->fmt == SNS_CSR_F32 || o->precondition == 0)) return SNS_EINVAL;
  return SNS_OK;
}

}  // namespace sns

using namespace sns;

extern "C" {

const char* snsolve_status_string(int s) {
  switch (s) {
    case SNS_OK: return "SNS_OK";
    case SNS_EINVAL: return "SNS_EINVAL";
    case SNS_ENOMEM: return "SNS_ENOMEM";
    case SNS_ERANK: return "SNS_ERANK";
    case SNS_ENOTCONV: return "SNS_ENOTCONV";
    case SNS_EAGAIN: return "SNS_EAGAIN";
    case SNS_ETIMEOUT: return "SNS_ETIMEOUT";
    case SNS_ECUDA: return "SNS_ECUDA";
    case SNS_EBUDGET: return "SNS_EBUDGET";
  }
  return "SNS_UNKNOWN";
}

const char* snsolve_last_cuda_error(void) { return t_err; }

int snsolve_version(void) { return 100; }

sns_status snsolve_create(sns_ctx** ctx, int device) {
  if (!ctx) return SNS_EINVAL;
  *ctx = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return record_cuda_error(e);
  if (device < 0 || device >= ndev) return SNS_EINVAL;
  int major = 0, minor = 0;
  SNS_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
  SNS_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
  if (major != 10 || minor != 3) {
    snprintf(t_err, sizeof(t_err), "device %d is sm_%d%d; this library is built for sm_103a", device, major, minor);
    return SNS_ECUDA;
  }
  int cur = 0;
  SNS_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != device) SNS_CUDA_TRY(cudaSetDevice(device));
  if (fault_hit(kFaultAlloc)) return record_injected("injected allocation failure", SNS_ENOMEM);
  sns_ctx* c = new sns_ctx();
  c->device = device;
  e = cudaHostAlloc(&c->pinned, 4096, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    delete c;
    return record_cuda_error(e);
  }
  memset(c->pinned, 0, 4096);
  *ctx = c;
  return SNS_OK;
}

void snsolve_destroy(sns_ctx* ctx) {
  if (!ctx) return;
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  delete ctx;
}

sns_status snsolve_sketch_workspace_size(const sns_problem* prob, const sns_sketch_desc* sk, size_t* bytes) {
  if (!bytes) return SNS_EINVAL;
  sns_status s = validate_problem(prob);
  if (s == SNS_OK) s = validate_sketch(prob, sk);
  if (s != SNS_OK) return s;
  *bytes = sketch_ws(prob, sk);
  return SNS_OK;
}

sns_status snsolve_sketch(sns_ctx* ctx, const sns_problem* prob, const sns_sketch_desc* sk, void* SA, int64_t ldsa,
                          void* Sb, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !SA || !Sb) return SNS_EINVAL;
  sns_status s = validate_problem(prob);
  if (s == SNS_OK) s = validate_sketch(prob, sk);
  if (s != SNS_OK) return s;
  if (ldsa < prob->n) return SNS_EINVAL;
  if (ws_bytes < sketch_ws(prob, sk) || (ws_bytes > 0 && !ws && sketch_ws(prob, sk) > 0)) return SNS_ENOMEM;
  if (ws && ((uintptr_t)ws % 256)) return SNS_EINVAL;
  return run_sketch(prob, sk, SA, ldsa, Sb, 1, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

sns_status snsolve_sketch_rows(sns_ctx* ctx, const sns_problem* prob, const sns_sketch_desc* sk, int64_t row0,
                               void* SA, int64_t ldsa, void* Sb, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !SA || !Sb) return SNS_EINVAL;
  sns_status s = validate_problem(prob);
  if (s == SNS_OK) s = validate_sketch(prob, sk);
  if (s != SNS_OK) return s;
  if (row0 < 0 || row0 > ((int64_t)1 << 40) || sk->kind == SNS_SRHT || ldsa < prob->n) return SNS_EINVAL;
  if (sk->kind == SNS_GAUSSIAN && row0 % 8 != 0) return SNS_EINVAL;   // one hash serves 8 consecutive rows
  if (ws_bytes < sketch_ws(prob, sk) || (ws_bytes > 0 && !ws && sketch_ws(prob, sk) > 0)) return SNS_ENOMEM;
  if (ws && ((uintptr_t)ws % 256)) return SNS_EINVAL;
  return run_sketch(prob, sk, SA, ldsa, Sb, 1, ws, ws_bytes, static_cast<cudaStream_t>(stream), row0);
}

// Workspace of snsolve_solve_sketched: FP64 column-major copy, status words,
// the multi-CTA QR's hand-off area.
struct SolveLayout {
  size_t off_w, off_dev, off_qr, bytes;
};
static SolveLayout solve_layout(int64_t d, int64_t n) {
  SolveLayout L{};
  const int64_t q = n + 1;
  size_t off = 0;
  L.off_w = off; off += al((size_t)d * q * 8);
  L.off_dev = off; off += al(64);
  L.off_qr = off; off += al(qr_coop_ws_bytes(d, q));
  L.bytes = off;
  return L;
}

sns_status snsolve_solve_sketched_workspace_size(int64_t d, int64_t n, size_t* bytes) {
  if (!bytes || n < 1 || d < n || d > 16384) return SNS_EINVAL;
  *bytes = solve_layout(d, n).bytes;
  return SNS_OK;
}

sns_status snsolve_solve_sketched(sns_ctx* ctx, const void* SAaug, int64_t ld, int32_t f64, int64_t d, int64_t n,
                                  double* x, sns_info* info, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !SAaug || !x || n < 1 || d < n || d > 16384 || ld < n + 1) return SNS_EINVAL;
  const SolveLayout L = solve_layout(d, n);
  if (!ws || ws_bytes < L.bytes) return SNS_ENOMEM;
  if ((uintptr_t)ws % 256) return SNS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w = static_cast<uint8_t*>(ws);
  const int64_t q = n + 1;
  double* W = reinterpret_cast<double*>(w + L.off_w);
  int32_t* dstatus = reinterpret_cast<int32_t*>(w + L.off_dev);
  double* dsres = reinterpret_cast<double*>(w + L.off_dev + 8);
  double* hp = thread_pinned();
  if (!hp) return SNS_ENOMEM;
  sns_status s = qr_load_colmajor(SAaug, ld, f64 != 0, d, q, W, st);
  if (s != SNS_OK) return s;
  QrOut o{W, d, q, x, dstatus, dsres};
  const bool coop = q >= 32;
  s = coop ? qr_solve_coop(o, w + L.off_qr, st) : qr_solve_one(o, st);
  if (s != SNS_OK) return s;
  SNS_CUDA_TRY(cudaMemcpyAsync(hp + 21, w + L.off_dev, 16, cudaMemcpyDeviceToHost, st));
  if (coop) SNS_CUDA_TRY(cudaMemcpyAsync(hp + 23, w + L.off_qr + qr_coop_err_offset(d, q), 4,
                                         cudaMemcpyDeviceToHost, st));
  SNS_CUDA_TRY(cudaStreamSynchronize(st));
  int32_t qs = 0, qerr = 0;
  memcpy(&qs, hp + 21, 4);
  if (coop) memcpy(&qerr, hp + 23, 4);
  if (fault_hit(kFaultTimeout)) qerr = 1;
  const int status = qerr ? SNS_ETIMEOUT : qs;
  if (info) {
    memset(info, 0, sizeof(*info));
    info->status = status;
    info->sketch_resid = qerr ? 0.0 : hp[22];
  }
  return (sns_status)status;
}

sns_status snsolve_sketch_status(const sns_problem* prob, const sns_sketch_desc* sk, const void* ws,
                                 size_t ws_bytes, void* stream) {
  sns_status s = validate_problem(prob);
  if (s == SNS_OK) s = validate_sketch(prob, sk);
  if (s != SNS_OK) return s;
  const void* word = sketch_err_word(prob, sk, static_cast<const uint8_t*>(ws));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!word) {
    SNS_CUDA_TRY(cudaStreamSynchronize(st));
    return SNS_OK;
  }
  if (!ws || ws_bytes < sketch_ws(prob, sk)) return SNS_EINVAL;
  double* hp = thread_pinned();
  if (!hp) return SNS_ENOMEM;
  SNS_CUDA_TRY(cudaMemcpyAsync(hp + 20, word, 4, cudaMemcpyDeviceToHost, st));
  SNS_CUDA_TRY(cudaStreamSynchronize(st));
  int32_t e = 0;
  memcpy(&e, hp + 20, 4);
  if (fault_hit(kFaultTimeout)) e = 1;
  return e ? SNS_ETIMEOUT : SNS_OK;
}

sns_status snsolve_lstsq_workspace_size(const sns_problem* prob, const sns_opts* opts, size_t* bytes) {
  if (!bytes) return SNS_EINVAL;
  sns_status s = validate_problem(prob);
  if (s == SNS_OK) s = validate_opts(prob, opts);
  if (s != SNS_OK) return s;
  *bytes = ls_layout(prob, opts).bytes;
  return SNS_OK;
}

static void info_fill(sns_info* info, int status, int iters, int outer, double eta, double rn, double sres) {
  if (!info) return;
  info->status = status;
  info->iters = iters;
  info->outer = outer;
  info->reserved = 0;
  info->eta = eta;
  info->resid_norm = rn;
  info->sketch_resid = sres;
  info->ms_sketch = info->ms_qr = info->ms_iter = 0.f;
  info->reserved2 = 0;
}

// Per-thread events bracketing a solve's phases on its stream: [0] start,
// [1] sketch done, [2] QR + back-solve done, [3] end.
struct PhaseEvents {
  cudaEvent_t e[4] = {};
  bool ok = false;
  int device = -1;
  ~PhaseEvents() {
    for (cudaEvent_t v : e)
      if (v) cudaEventDestroy(v);
  }
};
static thread_local PhaseEvents t_phase;
static PhaseEvents* phase_events() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (!t_phase.ok || t_phase.device != dev) {
    t_phase.ok = true;
    for (cudaEvent_t& v : t_phase.e)
      if (cudaEventCreate(&v) != cudaSuccess) t_phase.ok = false;
    t_phase.device = dev;
  }
  return t_phase.ok ? &t_phase : nullptr;
}
// Records the end event and fills the phase times of `info` (after info_fill).
static void phase_times(PhaseEvents* pe, cudaStream_t st, sns_info* info) {
  if (!pe || !info) return;
  if (cudaEventRecord(pe->e[3], st) != cudaSuccess || cudaEventSynchronize(pe->e[3]) != cudaSuccess) return;
  float t[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < 3; ++k)
    if (cudaEventElapsedTime(&t[k], pe->e[k], pe->e[k + 1]) != cudaSuccess) t[k] = 0.f;
  info->ms_sketch = t[0];
  info->ms_qr = t[1];
  info->ms_iter = t[2];
}

sns_status snsolve_lstsq(sns_ctx* ctx, const sns_problem* prob, const sns_opts* opts, double* x, sns_info* info,
                         void* ws, size_t ws_bytes, void* stream) {
  if (!ctx || !x) return SNS_EINVAL;
  sns_status s = validate_problem(prob);
  if (s == SNS_OK) s = validate_opts(prob, opts);
  if (s != SNS_OK) return s;
  const LsLayout L = ls_layout(prob, opts);
  if (!ws || ws_bytes < L.bytes) return SNS_ENOMEM;
  if ((uintptr_t)ws % 256) return SNS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint8_t* w = static_cast<uint8_t*>(ws);
  const int64_t n = prob->n, d = opts->sk.d, q = n + 1;
  const bool f64 = is_f64(prob);
  double* W = reinterpret_cast<double*>(w + L.off_w);
  int32_t* dstatus = reinterpret_cast<int32_t*>(w + L.off_dev);
  double* dsres = reinterpret_cast<double*>(w + L.off_dev + 8);
  double* hp = thread_pinned();
  if (!hp) return SNS_ENOMEM;
  const bool precond = opts->precondition != 0 || opts->tol <= 0;
  PhaseEvents* pe = phase_events();
  if (pe) SNS_CUDA_TRY(cudaEventRecord(pe->e[0], st));

  double sres = 0.0;
  if (precond) {
    // steps 1-2: S [A | b] into the augmented buffer (ld = n + 1)
    void* SA = w + L.off_saug;
    void* Sb = w + L.off_saug + (size_t)n * (f64 ? 8 : 4);
    const sns_sketch_desc sk = solve_sketch(opts);
    s = run_sketch(prob, &sk, SA, q, Sb, q, w + L.off_sk, L.sk_bytes, st);
    if (s != SNS_OK) return s;
    if (pe) SNS_CUDA_TRY(cudaEventRecord(pe->e[1], st));
    // step 3: FP64 Householder QR of [SA | Sb] and back substitution
    s = qr_load_colmajor(SA, q, f64, d, q, W, st);
    if (s != SNS_OK) return s;
    QrOut o{W, d, q, x, dstatus, dsres};
    const bool coop = q >= 32;
    s = coop ? qr_solve_coop(o, w + L.off_qr, st) : qr_solve_one(o, st);
    if (s != SNS_OK) return s;
    if (pe) SNS_CUDA_TRY(cudaEventRecord(pe->e[2], st));
    if (opts->tol > 0) {
      s = diag_range(W, d, n, reinterpret_cast<double*>(w + L.off_dev + 16), st);
      if (s != SNS_OK) return s;
      SNS_CUDA_TRY(cudaMemcpyAsync(hp + 24, w + L.off_dev + 16, 16, cudaMemcpyDeviceToHost, st));
    }
    SNS_CUDA_TRY(cudaMemcpyAsync(hp + 16, w + L.off_dev, 16, cudaMemcpyDeviceToHost, st));
    if (coop) {
      const size_t eoff = L.off_qr + qr_coop_err_offset(d, q);
      SNS_CUDA_TRY(cudaMemcpyAsync(hp + 18, w + eoff, 4, cudaMemcpyDeviceToHost, st));
    }
    const void* skerr = sketch_err_word(prob, &sk, w + L.off_sk);
    if (skerr) SNS_CUDA_TRY(cudaMemcpyAsync(hp + 19, skerr, 4, cudaMemcpyDeviceToHost, st));
    SNS_CUDA_TRY(cudaStreamSynchronize(st));
    int32_t qs, qerr = 0, serr = 0;
    memcpy(&qs, hp + 16, 4);
    if (coop) memcpy(&qerr, hp + 18, 4);
    if (skerr) memcpy(&serr, hp + 19, 4);
    if (fault_hit(kFaultTimeout)) serr = 1;
    sres = hp[17];
    if (qerr || serr) {
      info_fill(info, SNS_ETIMEOUT, 0, 0, 0.0, 0.0, 0.0);
      phase_times(pe, st, info);
      return SNS_ETIMEOUT;
    }
    if (qs != SNS_OK) {
      info_fill(info, qs, 0, 0, 0.0, 0.0, sres);
      phase_times(pe, st, info);
      return (sns_status)qs;
    }
    if (opts->tol <= 0) {
      info_fill(info, SNS_OK, 0, 0, 0.0, 0.0, sres);
      phase_times(pe, st, info);
      return SNS_OK;
    }
  } else {
    if (pe) {
      SNS_CUDA_TRY(cudaEventRecord(pe->e[1], st));
      SNS_CUDA_TRY(cudaEventRecord(pe->e[2], st));
    }
    SNS_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)n * 8, st));
  }

  // SAP-SAS refinement.  R^{-1} is built on a side stream while the first
  // residual pass (which only needs x) runs on the caller's stream.
  const IterWs I = iter_ws_carve(w + L.off_iter, n, L.grid);
  SNS_CUDA_TRY(cudaMemsetAsync(I.ticket, 0, 64 * 4, st));
  SideStream& side = thread_side_stream();
  if (!side.ok) return SNS_ECUDA;
  SNS_CUDA_TRY(cudaEventRecord(side.ev_in, st));
  SNS_CUDA_TRY(cudaStreamWaitEvent(side.st, side.ev_in, 0));
  const bool saa = uses_saa(opts);
  const bool factored = precond && !saa && hp[25] > 0.0 && hp[24] > kFactoredDiagRatio * hp[25];
  s = rinv_build(W, d, n, I.Rinv, I.RinvT, !precond, side.st);
  if (s != SNS_OK) return s;
  // SAP: M^-1 = R^-1 R^-T in x-space (formed, or factored); SAA: CG on Y^T Y in z-space, M = I
  if (saa) s = ident_build(I.P, n, side.st);
  else if (!factored) s = pgram_build(I.Rinv, n, I.P, side.st);
  if (s != SNS_OK) return s;
  SNS_CUDA_TRY(cudaEventRecord(side.ev_out, side.st));
  bool rinv_joined = false;
  DenseArgs da{prob->A, prob->lda, prob->b, prob->m, n, f64};
  CsrArgs ca{prob->rowptr, prob->col, prob->val, static_cast<const float*>(prob->b), prob->m, n, prob->nnz};
  ca.det = opts->sk.kind == SNS_COUNTSKETCH && opts->sk.variant == SNS_CS_SORTED;   // reproducible CSR solve
  const DenseArgs* dap = prob->fmt == SNS_CSR_F32 ? nullptr : &da;
  const CsrArgs* cap = prob->fmt == SNS_CSR_F32 ? &ca : nullptr;
  // SAA: the explicit Y = A R^-1, formed before the first inner cycle
  void* Y = w + L.off_y;
  const DenseArgs ya{Y, saa_ldy(n, f64), nullptr, prob->m, n, f64};
  bool y_ready = false;
  const int max_iter = opts->max_iter > 0 ? opts->max_iter : 400;
  const int inner = opts->inner > 0 ? opts->inner : kDefaultInnerMax;
  int passes = 0, outer = 0, passes_before = -1;
  double eta = 0.0, rn = 0.0;
  s = iter_reset(I, st);
  if (s != SNS_OK) return s;
  for (;;) {
    s = resid_pass(dap, cap, x, I, outer == 0, opts->tol < kCheapGradTol, st);
    if (s != SNS_OK) return s;
    s = eta_eval(I, n, hp, st);
    if (s != SNS_OK) return s;
    SNS_CUDA_TRY(cudaStreamSynchronize(st));
    ++outer;
    eta = hp[0];
    rn = hp[1];
    passes = (int)hp[4];                 // normal passes the cycles actually ran
    if (!(eta > opts->tol)) break;       // converged (also stops on eta == 0)
    if (outer > 1 && passes == passes_before) {
      // the last cycle could not take a single step (its preconditioned
      // residual was not positive): no further progress is possible
      if (!rinv_joined) SNS_CUDA_TRY(cudaStreamWaitEvent(st, side.ev_out, 0));
      info_fill(info, SNS_ENOTCONV, passes, outer, eta, rn, sres);
      phase_times(pe, st, info);
      return SNS_ENOTCONV;
    }
    if (passes >= max_iter) {
      if (!rinv_joined) SNS_CUDA_TRY(cudaStreamWaitEvent(st, side.ev_out, 0));
      info_fill(info, SNS_ENOTCONV, passes, outer, eta, rn, sres);
      phase_times(pe, st, info);
      return SNS_ENOTCONV;
    }
    // inner solver: preconditioned CG on A^T A dx = g (M^-1 = R^-1 R^-T); the
    // cycle stops itself on the device, later launches of the budget return at once
    if (!rinv_joined) {
      SNS_CUDA_TRY(cudaStreamWaitEvent(st, side.ev_out, 0));
      rinv_joined = true;
    }
    if (saa) {
      if (!y_ready) {
        if ((s = saa_form_y(da, I.Rinv, Y, st)) != SNS_OK) return s;
        y_ready = true;
      }
      // right-hand side Y^T r = R^-T g (into w, which the first pass overwrites)
      if ((s = saa_matvec(I.RinvT, n, I.g, I.w, false, st)) != SNS_OK) return s;
      s = pcg_start_rhs(I, n, opts->tol, I.w, st);
    } else {
      s = pcg_start(I, n, opts->tol, st, factored);
    }
    if (s != SNS_OK) return s;
    const int budget = std::min(inner, max_iter - passes);
    for (int k = 0; k < budget; ++k) {
      if ((s = saa ? normal_pass(&ya, nullptr, I, st) : normal_pass(dap, cap, I, st)) != SNS_OK) return s;
      if ((s = pcg_step(I, n, st, factored)) != SNS_OK) return s;
    }
    passes_before = passes;
    // x += dx (SAP), x += R^-1 dz (SAA)
    s = saa ? saa_matvec(I.Rinv, n, I.dx, x, true, st) : pcg_apply(I, n, x, st);
    if (s != SNS_OK) return s;
  }
  if (!rinv_joined) SNS_CUDA_TRY(cudaStreamWaitEvent(st, side.ev_out, 0));
  info_fill(info, SNS_OK, passes, outer, eta, rn, sres);
  phase_times(pe, st, info);
  return SNS_OK;
}

// ---------------------------------------------------------------- batched
sns_status snsolve_lstsq_batched_workspace_size(const sns_problem* probs, const sns_opts* opts, int nprob,
                                                size_t* bytes) {
  if (!bytes || !probs || !opts || nprob < 1) return SNS_EINVAL;
  for (int i = 0; i < nprob; ++i) {
    sns_status s = validate_problem(probs + i);
    if (s == SNS_OK) s = validate_opts(probs + i, opts + i);
    if (s != SNS_OK) return s;
  }
  *bytes = batch_ws_bytes(probs, opts, nprob);
  return SNS_OK;
}

sns_status snsolve_lstsq_batched(sns_ctx* ctx, const sns_problem* probs, const sns_opts* opts, int nprob,
                                 double* const* x, sns_info* infos, void* ws, size_t ws_bytes, void* stream) {
  if (!ctx) return SNS_EINVAL;
  return lstsq_batched(probs, opts, nprob, x, infos, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------- debug ABI
sns_status snsolve_debug_countsketch_hash(int64_t m, int64_t d, uint64_t seed, uint32_t* h, int8_t* s, void* stream) {
  if (m < 0 || d < 1 || !h || !s) return SNS_EINVAL;
  return debug_countsketch_hash(m, d, seed, h, s, static_cast<cudaStream_t>(stream));
}
sns_status snsolve_debug_stream_keys(uint64_t seed, int stream_id, int64_t start, int64_t count, uint64_t* keys,
                                     void* stream) {
  if (count < 0 || start < 0 || !keys || stream_id < 0 || stream_id > 255) return SNS_EINVAL;
  return debug_stream_keys(seed, stream_id, start, count, keys, static_cast<cudaStream_t>(stream));
}
sns_status snsolve_debug_srht_sample(int64_t mp, int64_t d, uint64_t seed, int64_t* idx, void* ws, size_t ws_bytes,
                                     void* stream) {
  if (mp < 1 || (mp & (mp - 1)) || d < 1 || d > mp || !idx || mp >= ((int64_t)1 << 31)) return SNS_EINVAL;
  return debug_srht_sample(mp, d, seed, idx, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}
sns_status snsolve_debug_srht_sample_ws(int64_t mp, int64_t d, size_t* bytes) {
  if (!bytes || mp < 1 || d < 1) return SNS_EINVAL;
  const size_t m2 = (size_t)(mp < 1024 ? mp : 1024);
  *bytes = ((size_t)d * 4 + 255) / 256 * 256 + (m2 + 255) / 256 * 256 + (m2 + 1) * 4;
  return SNS_OK;
}
void snsolve_debug_set_qr_wait_limit(int64_t polls) { set_qr_wait_limit((long long)polls); }

sns_status snsolve_debug_set_fault(const char* spec) { return fault_arm(spec); }

int snsolve_debug_fault_armed(int64_t* left) {
  long long l = 0;
  const int k = fault_armed(&l);
  if (left) *left = (int64_t)l;
  return k;
}

sns_status snsolve_debug_form_y(const sns_problem* prob, const double* Rinv, void* Y, int64_t ldy, void* stream) {
  sns_status s = validate_problem(prob);
  if (s != SNS_OK) return s;
  if (prob->fmt == SNS_CSR_F32 || !Rinv || !Y || ldy < prob->n) return SNS_EINVAL;
  DenseArgs da{prob->A, prob->lda, prob->b, prob->m, prob->n, is_f64(prob)};
  return saa_form_y(da, Rinv, Y, static_cast<cudaStream_t>(stream), ldy);
}

sns_status snsolve_debug_gaussian_table(uint16_t* bf16_bits_host) {
  if (!bf16_bits_host) return SNS_EINVAL;
  gauss_table_host(bf16_bits_host);
  return SNS_OK;
}

}  // extern "C"
