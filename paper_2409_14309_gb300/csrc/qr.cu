// FP64 Householder QR of the sketched augmented matrix [SA | Sb] (d x (n+1)) and
// the triangular solves of sketch-and-solve (Sec. 1.2 step 3, which leaves the
// small problem to standard solvers; the reduced problem of Sec. 1.3).
//
// R_aug = the (n+1) x (n+1) triangular factor of [SA | Sb]: its leading n x n
// block is R, its last column holds z = (Q^T Sb)[0:n], and |R_aug[n, n]| is the
// sketched residual ||SA x^ - Sb||.  x^ = R^{-1} z.
//
// Reflector convention: for column x (rows j..d-1), alpha = -sign(x_0) ||x||
// (x_0 = 0 counts as positive), v = x - alpha e_0 scaled so v_0 = 1,
// tau = -v_0 / alpha; R[j, j] = alpha.
#include <cuda_runtime.h>

#include <atomic>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"
#include "qr_cta.cuh"

namespace sns {

constexpr int kQrThreads = 256;

template <typename T>
__global__ void qr_load_kernel(const T* __restrict__ S, int64_t ld, int64_t d, int64_t q, double* __restrict__ W) {
  const int64_t total = d * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / q, c = e % q;
    W[c * d + r] = (double)S[r * ld + c];
  }
}

sns_status qr_load_colmajor(const void* SAaug, int64_t ld, bool f64, int64_t d, int64_t q, double* W, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>((d * q + 255) / 256, (int64_t)num_sms() * 8);
  if (f64)
    {
      SNS_PROF(K_QR_LOAD, st);
    qr_load_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(SAaug), ld, d, q, W);
    }
  else
    {
      SNS_PROF(K_QR_LOAD, st);
    qr_load_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(SAaug), ld, d, q, W);
    }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

__global__ void __launch_bounds__(kQrThreads) qr_tasks_kernel(const QrOut* __restrict__ tasks, int ntasks) {
  extern __shared__ double qsm[];
  __shared__ double red[32];
  for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
    const QrOut o = tasks[t];
    double* v = qsm;                 // d entries
    qr_factor_cta(o.W, o.d, o.q, v, red);
    qr_finish_cta(o.W, o.d, o.q, o.x, o.status, o.sres, qsm, red);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kQrThreads) qr_one_kernel(QrOut o) {
  extern __shared__ double qsm[];
  __shared__ double red[32];
  qr_factor_cta(o.W, o.d, o.q, qsm, red);
  qr_finish_cta(o.W, o.d, o.q, o.x, o.status, o.sres, qsm, red);
}

sns_status qr_solve_one(const QrOut& o, cudaStream_t st) {
  const size_t smem = (size_t)std::max<int64_t>(o.d, 2 * o.q) * 8;
  SNS_CUDA_TRY(raise_smem_limit((const void*)qr_one_kernel));
  {
    SNS_PROF(K_QR, st);
  qr_one_kernel<<<1, kQrThreads, smem, st>>>(o);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

sns_status qr_solve_tasks(const QrOut* tasks_dev, int ntasks, int64_t max_d, cudaStream_t st) {
  const size_t smem = (size_t)(2 * max_d + 2) * 8;     // factor: d doubles; finish: 2 q <= 2 d + 2
  SNS_CUDA_TRY(raise_smem_limit((const void*)qr_tasks_kernel));
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, qr_tasks_kernel, kQrThreads, smem));
  const int grid = std::min(ntasks, num_sms() * std::max(occ, 1));
  {
    SNS_PROF(K_QR, st);
  qr_tasks_kernel<<<grid, kQrThreads, smem, st>>>(tasks_dev, ntasks);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

// ---------------------------------------------------------------------------
// Multi-CTA Householder QR for one large problem (cooperative launch, all CTAs
// resident).  Column c belongs to CTA c mod G and, when the owned columns fit,
// lives in that CTA's shared memory for the whole factorisation.
//
// Reflector j is published unscaled: u_j = x - alpha e_0 over rows j..d-1
// (u_j[0] = x_0 - alpha = v_0), H_j = I - beta_j u_j u_j^T with
// beta_j = tau_j / v_0^2 = -1 / (alpha v_0), which is the same H as the
// (v_0 = 1, tau) form without the scaling pass.  Rows j+1.. of u_j go to
// U[j, j+1:] and (beta_j, v_0) to pub[j].
//
// Hand-off without flags: U and pub are filled with an all-ones bit pattern
// (a NaN that no arithmetic produces; a computed value with that pattern is
// published as the canonical NaN) before the launch, and every consumer thread
// polls exactly the values it needs until they differ from it.  Each value
// validates itself, so the producer needs no fence and the consumer no flag
// round trip: one L2 trip per hand-off.
//
// GB300's FP64 pipe issues about half a lane per clock per SM sub-partition,
// so the kernel keeps FP64 instructions off the serial chain: 128 threads (one
// warp per sub-partition), a fixed row-to-thread map so a thread uses only the
// reflector rows it loaded itself, scalar work (sqrt, divide) on one thread,
// and one batched reduction per step for the non-critical columns.
// Look-ahead: the owner of column j+1 updates it with reflector j, builds and
// publishes reflector j+1, and only then updates its other columns.  Waits
// are bounded: after kSpinLimit polls a thread records an error and carries on
// with zeros; later waits see the error word and stop polling, so a failed
// factorisation ends quickly and the host reports it.
constexpr long long kSpinLimit = 1LL << 22;
// Poll limit of the next cooperative factorisations (0: kSpinLimit); set by
// snsolve_debug_set_qr_wait_limit to exercise the timeout path.
static std::atomic<long long> g_qr_wait_limit{0};
void set_qr_wait_limit(long long polls) { g_qr_wait_limit.store(polls > 0 ? polls : 0, std::memory_order_relaxed); }
constexpr int kCoopThreads = 128;
constexpr int kCoopWarps = kCoopThreads / 32;
constexpr int kCoopBatch = 8;                 // non-critical columns per batched reduction
constexpr long long kSentinel = -1LL;         // all-ones bit pattern: "not yet published"

SNS_D double ld_relaxed(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
SNS_D int ld_relaxed_int(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
SNS_D void st_relaxed(double* p, double v) {
  if (__double_as_longlong(v) == kSentinel) v = __longlong_as_double(0x7FF8000000000000LL);
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Polls up to kSlots addresses (null = unused) until none holds the sentinel;
// bounded as described above.
template <int kSlots>
SNS_D void coop_poll(const double* const (&addr)[kSlots], double (&val)[kSlots], int* err, long long limit) {
  bool got[kSlots];
#pragma unroll
  for (int u = 0; u < kSlots; ++u) got[u] = (addr[u] == nullptr);
  for (long long it = 0;; ++it) {
    bool all = true;
#pragma unroll
    for (int u = 0; u < kSlots; ++u)
      if (!got[u]) {
        val[u] = ld_relaxed(addr[u]);
        got[u] = __double_as_longlong(val[u]) != kSentinel;
        all = all && got[u];
      }
    if (all) return;
    const bool give_up = it >= limit;
    if (give_up || ((it & 255) == 255 && ld_relaxed_int(err) != 0)) {
      if (give_up) atomicExch(err, 1);
#pragma unroll
      for (int u = 0; u < kSlots; ++u)
        if (!got[u]) val[u] = 0.0;
      return;
    }
    if (it >= 4096) __nanosleep(32);
  }
}

// Sum over the CTA of one value per thread; thread 0 receives the total
// (other threads receive garbage).  Two reductions in a row are safe: thread 0
// reads red[] before the barrier that the next writers must pass.
SNS_D double coop_sum0(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < kCoopWarps; ++w) t += red[w];
  }
  return t;
}

// Same sum, every thread receives it (one barrier; each thread adds the
// kCoopWarps partials in the same order).
SNS_D double coop_sum_all(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kCoopWarps; ++w) t += red[w];
  return t;
}

// First row >= j of this thread's fixed residue class (rows i = tid mod T).
SNS_D int64_t coop_first_row(int64_t j) {
  return j + (int64_t)((threadIdx.x - (int)(j % kCoopThreads) + kCoopThreads) % kCoopThreads);
}

// Applies reflector j (rows j.., this thread's rows of vsm; scale beta) to CNT
// owned columns c0, c0 + cstride, ...: one batched CTA reduction for all dots.
template <int CNT>
SNS_D void coop_batch(double* c0, int64_t cstride, int64_t d, int64_t j, double beta, const double* vsm,
                      double (*red)[kCoopWarps], double* bcast) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double part[CNT];
#pragma unroll
  for (int t = 0; t < CNT; ++t) part[t] = 0.0;
  for (int64_t i = coop_first_row(j); i < d; i += kCoopThreads) {
    const double vi = vsm[i];
#pragma unroll
    for (int t = 0; t < CNT; ++t) part[t] = fma(vi, c0[t * cstride + i], part[t]);
  }
#pragma unroll
  for (int t = 0; t < CNT; ++t) {
    const double ws = warp_sum(part[t]);
    if (lane == 0) red[t][wid] = ws;
  }
  __syncthreads();
  if (tid < CNT) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kCoopWarps; ++w) s += red[tid][w];
    bcast[tid] = beta * s;
  }
  __syncthreads();
  double f[CNT];
#pragma unroll
  for (int t = 0; t < CNT; ++t) f[t] = bcast[t];
  for (int64_t i = coop_first_row(j); i < d; i += kCoopThreads) {
    const double vi = vsm[i];
#pragma unroll
    for (int t = 0; t < CNT; ++t) c0[t * cstride + i] = fma(-f[t], vi, c0[t * cstride + i]);
  }
}

template <bool kSmemCols>
__global__ void __launch_bounds__(kCoopThreads, 1)
qr_coop_kernel(double* __restrict__ W, int64_t d, int64_t q, double* __restrict__ U, double* __restrict__ pub,
               int* __restrict__ err, long long spin_limit) {
  extern __shared__ __align__(16) double qsm[];
  double* vsm = qsm;                                   // reflector rows (fixed row map)
  double* csm = qsm + d;                               // owned columns (kSmemCols)
  __shared__ double red[kCoopBatch][kCoopWarps];     // batched reductions
  __shared__ double redc[2][kCoopWarps];             // the critical column's two reductions
  __shared__ double bcast[kCoopBatch + 4];
  const int tid = threadIdx.x;
  const int64_t G = gridDim.x, b = blockIdx.x;
  const int64_t steps = q < d ? q : d;
  if (b >= q) return;
  const int64_t nown = (q - 1 - b) / G + 1;
  const int64_t clast = b + (nown - 1) * G;
  auto col = [&](int64_t k) -> double* { return kSmemCols ? csm + k * d : W + (b + k * G) * d; };
  const int64_t cstride = kSmemCols ? d : G * d;       // distance between consecutive owned columns
  if (kSmemCols) {
    for (int64_t k = 0; k < nown; ++k) {
      const double* src = W + (b + k * G) * d;
      for (int64_t i = tid; i < d; i += kCoopThreads) csm[k * d + i] = src[i];
    }
    __syncthreads();
  }

  // Update column cc with reflector j (rows >= j; f = beta * u^T c), then
  // build reflector c1 = j + 1 from it and publish.  With j < 0 the column is
  // only reflected (column 0).  The dot over rows > j and its CTA reduction
  // need neither beta nor v_0 (row j's u entry), so they run before
  // scalars() fetches them: the reflector's rows are published ahead of its
  // scalars, and this overlaps the dot with the producer's norm and sqrt.
  auto critical = [&](double* cc, int64_t j, auto&& scalars, double& beta, double& v0) {
    const int64_t c1 = j + 1;
    double f = 0.0;
    if (j >= 0) {
      // early, non-blocking tries at beta_j and v_0: the poll below costs a
      // full L2 round trip when it starts only after the reduction
      const double* ps = pub + 2 * j;
      const double e0b = ld_relaxed(ps), e0v = ld_relaxed(ps + 1);
      double part = 0.0;
      for (int64_t i = coop_first_row(j + 1); i < d; i += kCoopThreads) part = fma(vsm[i], cc[i], part);
      const double e1b = ld_relaxed(ps), e1v = ld_relaxed(ps + 1);
      // row j of this column, read by every thread before the reduction's
      // barrier: its owner overwrites it in the update loop below
      const double cj = cc[j];
      const double t = coop_sum_all(part, redc[0]);
      scalars(e0b, e0v, e1b, e1v);
      if (beta != 0.0) f = beta * fma(v0, cj, t);
    }
    const bool publish = c1 < steps;
    double* ucol = U + c1 * d;                         // published rows c1+1..
    double nrm = 0.0;
    const int64_t i0 = coop_first_row(j >= 0 ? j : 0);
    for (int64_t i = i0; i < d; i += kCoopThreads) {
      double c = cc[i];
      if (f != 0.0) {
        c = fma(-f, vsm[i], c);
        cc[i] = c;
      }
      if (i >= c1) nrm = fma(c, c, nrm);
      if (publish && i > c1) st_relaxed(ucol + i, c);
    }
    if (!publish) return;                              // no reflector for this column
    const double nrm2 = coop_sum0(nrm, redc[1]);
    if (tid == 0) {
      const double x0 = cc[c1];
      const double normx = sqrt(nrm2);
      double alpha = x0, vv0 = 0.0, bt = 0.0;
      if (normx > 0.0) {
        alpha = (x0 >= 0.0) ? -normx : normx;
        vv0 = x0 - alpha;
        bt = -1.0 / (alpha * vv0);
      }
      cc[c1] = alpha;
      bcast[kCoopBatch + 1] = bt;
      bcast[kCoopBatch + 2] = vv0;
      st_relaxed(pub + 2 * c1, bt);
      st_relaxed(pub + 2 * c1 + 1, vv0);
    }
  };

  {
    double b0 = 0.0, v00 = 0.0;
    if (b == 0) critical(col(0), -1, [](double, double, double, double) {}, b0, v00);
  }
  const int64_t jend = clast < steps ? clast : steps;
  for (int64_t j = 0; j < jend; ++j) {
    const bool mine = (j % G) == b;
    __syncthreads();                                   // previous step done; owner's bcast visible
    // reflector j's rows > j into this thread's rows of vsm
    double beta = 0.0, v0 = 0.0;
    const bool row_j = coop_first_row(j) == j;         // this thread holds row j (u_j[0] = v_0)
    if (mine) {
      beta = bcast[kCoopBatch + 1];
      v0 = bcast[kCoopBatch + 2];
      const double* cj = col((j - b) / G);
      for (int64_t i = coop_first_row(j + 1); i < d; i += kCoopThreads) vsm[i] = cj[i];
    } else {
      const double* uj = U + j * d;
      for (int64_t i = coop_first_row(j + 1); i < d; i += 8 * kCoopThreads) {
        const double* ad[8];
        double vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) ad[u] = (i + u * kCoopThreads < d) ? uj + i + u * kCoopThreads : nullptr;
        coop_poll<8>(ad, vv, err, spin_limit);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (ad[u]) vsm[i + u * kCoopThreads] = vv[u];
      }
    }
    // beta_j and v_0 (published after the rows; the caller may pass two
    // earlier loads of them, used if either already holds the values); row j
    // of vsm
    auto scalars = [&](double e0b, double e0v, double e1b, double e1v) {
      if (!mine) {
        auto ready = [](double x) { return __double_as_longlong(x) != kSentinel; };
        if (ready(e0b) && ready(e0v)) {
          beta = e0b;
          v0 = e0v;
        } else if (ready(e1b) && ready(e1v)) {
          beta = e1b;
          v0 = e1v;
        } else {
          const double* ad[2] = {pub + 2 * j, pub + 2 * j + 1};
          double vv[2];
          coop_poll<2>(ad, vv, err, spin_limit);
          beta = vv[0];
          v0 = vv[1];
        }
      }
      if (row_j) vsm[j] = v0;
    };
    // look-ahead column j + 1
    const int64_t c1 = j + 1;
    const double none = __longlong_as_double(kSentinel);
    if (c1 % G == b) critical(col((c1 - b) / G), j, scalars, beta, v0);
    else scalars(none, none, none, none);
    if (beta == 0.0) continue;
    // other owned columns > j + 1, up to kCoopBatch per batched reduction
    int64_t k0 = (c1 + 1 - b + G - 1) / G;               // first owned index with column > j + 1
    if (c1 + 1 <= b) k0 = 0;
    for (; k0 < nown; k0 += kCoopBatch) {
      const int cnt = (int)((nown - k0) < kCoopBatch ? (nown - k0) : kCoopBatch);
      switch (cnt) {   // compile-time column counts: no predicated-off FP64 instructions
        case 1: coop_batch<1>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
        case 2: coop_batch<2>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
        case 3: coop_batch<3>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
        case 4: coop_batch<4>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
        case 5: coop_batch<5>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
        case 6: coop_batch<6>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
        case 7: coop_batch<7>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
        default: coop_batch<8>(col(k0), cstride, d, j, beta, vsm, red, bcast); break;
      }
    }
  }
  if (kSmemCols) {
    __syncthreads();
    for (int64_t k = 0; k < nown; ++k) {
      double* dst = W + (b + k * G) * d;
      for (int64_t i = tid; i < d; i += kCoopThreads) dst[i] = csm[k * d + i];
    }
  }
}

// Rank check + back substitution of a factorised problem on one CTA.
constexpr int kFinishThreads = 128;
constexpr int kTriRing = 8;
__global__ void __launch_bounds__(kFinishThreads) qr_finish_kernel(QrOut o) {
  extern __shared__ __align__(16) double zsm[];
  __shared__ double red[32];
  qr_finish_cta<kTriRing>(o.W, o.d, o.q, o.x, o.status, o.sres, zsm, red);
}

// Up to two CTAs per SM: with fewer columns per CTA, the CTA about to build the
// next reflector has no other columns' updates queued in front of it (measured:
// 4.33 -> 4.15 us per column at d = 1024, q = 257; 7.9 -> 6.9 at d = 2048,
// q = 513).  The launcher checks co-residency.
static int qr_coop_grid(int64_t q) { return (int)std::max<int64_t>(1, std::min<int64_t>(q, 2 * (int64_t)num_sms())); }

// Workspace: U (q x d doubles) | pub (2 q doubles) | err (int).  U and pub are
// set to the sentinel and err to 0 by one memset each per factorisation.
static size_t qr_coop_sent_bytes(int64_t d, int64_t q) { return (size_t)q * d * 8 + (size_t)q * 16; }
size_t qr_coop_ws_bytes(int64_t d, int64_t q) { return ((qr_coop_sent_bytes(d, q) + 255) & ~(size_t)255) + 256; }
size_t qr_coop_err_offset(int64_t d, int64_t q) { return (qr_coop_sent_bytes(d, q) + 255) & ~(size_t)255; }

sns_status qr_solve_coop(const QrOut& o, void* ws, cudaStream_t st) {
  uint8_t* w = static_cast<uint8_t*>(ws);
  double* U = reinterpret_cast<double*>(w);
  double* pub = U + (size_t)o.q * o.d;
  int* err = reinterpret_cast<int*>(w + qr_coop_err_offset(o.d, o.q));
  SNS_CUDA_TRY(cudaMemsetAsync(U, 0xFF, qr_coop_sent_bytes(o.d, o.q), st));
  SNS_CUDA_TRY(cudaMemsetAsync(err, 0, 4, st));
  int dev = 0, smem_max = 0;
  SNS_CUDA_TRY(cudaGetDevice(&dev));
  SNS_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t static_smem = 2048;                     // red, bcast (upper bound)
  // widest grid (up to two CTAs per SM) whose CTAs are all co-resident
  int grid = 0;
  size_t smem = 0;
  const void* fn = nullptr;
  for (int g = qr_coop_grid(o.q); g >= 1; g = (g > num_sms()) ? num_sms() : 0) {
    const int64_t own = (o.q + g - 1) / g;
    const size_t smem_cols = (size_t)(1 + own) * o.d * 8;
    const bool in_smem = smem_cols + static_smem <= (size_t)smem_max;
    const size_t sm = in_smem ? smem_cols : (size_t)o.d * 8;
    const void* f = in_smem ? (const void*)qr_coop_kernel<true> : (const void*)qr_coop_kernel<false>;
    SNS_CUDA_TRY(raise_smem_limit(f));
    int occ = 0;
    SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kCoopThreads, sm));
    if ((int64_t)occ * num_sms() >= g) {
      grid = g;
      smem = sm;
      fn = f;
      break;
    }
  }
  if (!fn) return SNS_EINVAL;
  double* W = o.W;
  int64_t d = o.d, q = o.q;
  long long limit = g_qr_wait_limit.load(std::memory_order_relaxed);
  if (limit <= 0) limit = kSpinLimit;
  void* args[] = {&W, &d, &q, &U, &pub, &err, &limit};
  {
    SNS_PROF(K_QR, st);
    SNS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kCoopThreads), args, smem, st));
  }
  const size_t zs = (size_t)std::max<int64_t>(o.q, 1) * 8 * (2 + kTriRing);
  SNS_CUDA_TRY(raise_smem_limit((const void*)qr_finish_kernel));
  {
    SNS_PROF(K_QR, st);
    qr_finish_kernel<<<1, kFinishThreads, zs, st>>>(o);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

// Explicit R^{-1} (upper triangular, FP64) for the preconditioner applications
// of the iterative phase.  One CTA per column j solves R y = e_j by
// column-oriented back substitution (tri_backsolve_cta: reciprocal diagonal,
// one barrier per step, R's columns streamed ahead through a cp.async ring);
// the longest columns are scheduled first.  Writes Rinv (row-major) and its
// transpose RinvT (row-major).  With `identity`, writes the identity
// (unpreconditioned iteration).
constexpr int kRinvThreads = 128;
__global__ void __launch_bounds__(kRinvThreads) rinv_kernel(const double* __restrict__ W, int64_t ldw, int64_t n,
                                                            double* __restrict__ Rinv, double* __restrict__ RinvT,
                                                            int identity) {
  extern __shared__ __align__(16) double rsm[];
  double* ycol = rsm;                 // n
  double* rd = rsm + n;               // n: 1 / R[k, k]
  double* ring = rsm + 2 * n;         // kTriRing columns
  if (!identity)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) rd[i] = 1.0 / W[i * ldw + i];
  for (int64_t jj = blockIdx.x; jj < n; jj += gridDim.x) {
    const int64_t j = n - 1 - jj;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) ycol[i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    if (!identity) {
      tri_backsolve_cta<kTriRing>(W, ldw, j, ycol, rd, ring, n, [&](int64_t k, double yk) {
        Rinv[k * n + j] = yk;
        RinvT[j * n + k] = yk;
      });
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      if (identity || i > j) {
        const double v = (i == j) ? 1.0 : 0.0;
        Rinv[i * n + j] = v;
        RinvT[j * n + i] = v;
      }
    }
    __syncthreads();
  }
}

sns_status rinv_build(const double* W, int64_t ldw, int64_t n, double* Rinv, double* RinvT, bool identity,
                      cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, 4096));
  const size_t smem = (size_t)n * 8 * (2 + kTriRing);
  SNS_CUDA_TRY(raise_smem_limit((const void*)rinv_kernel));
  {
    SNS_PROF(K_RINV, st);
    rinv_kernel<<<grid, kRinvThreads, smem, st>>>(W, ldw, n, Rinv, RinvT, identity ? 1 : 0);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

}  // namespace sns
