// FP64 Householder QR of the sketched augmented matrix [SA | Sb] (d x (n+1)) and
// the triangular solves of sketch-and-solve (Sec. 1.2 step 3: "solve on SA
// using existing algorithms"; the reduced problem of Sec. 1.3).
//
// R_aug = the (n+1) x (n+1) triangular factor of [SA | Sb]: its leading n x n
// block is R, its last column holds z = (Q^T Sb)[0:n], and |R_aug[n, n]| is the
// sketched residual ||SA x^ - Sb||.  x^ = R^{-1} z.
//
// Reflector convention: for column x (rows j..d-1), alpha = -sign(x_0) ||x||
// (x_0 = 0 counts as positive), v = x - alpha e_0 scaled so v_0 = 1,
// tau = -v_0 / alpha; R[j, j] = alpha.
#include <cuda_runtime.h>
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
  SNS_CUDA_TRY(cudaGetLastError());
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
  const size_t smem = (size_t)std::max<int64_t>(o.d, o.q) * 8;
  SNS_CUDA_TRY(raise_smem_limit((const void*)qr_one_kernel));
  {
    SNS_PROF(K_QR, st);
  qr_one_kernel<<<1, kQrThreads, smem, st>>>(o);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

sns_status qr_solve_tasks(const QrOut* tasks_dev, int ntasks, int64_t max_d, cudaStream_t st) {
  const size_t smem = (size_t)max_d * 8;
  SNS_CUDA_TRY(raise_smem_limit((const void*)qr_tasks_kernel));
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, qr_tasks_kernel, kQrThreads, smem));
  const int grid = std::min(ntasks, num_sms() * std::max(occ, 1));
  {
    SNS_PROF(K_QR, st);
  qr_tasks_kernel<<<grid, kQrThreads, smem, st>>>(tasks_dev, ntasks);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

// ---------------------------------------------------------------------------
// Multi-CTA Householder QR for one large problem (cooperative launch, all CTAs
// resident).  Column c belongs to CTA c mod G.  Reflector j is published by the
// owner of column j: v_j overwrites W[j+1:, j] (v_j[0] = 1 implicit), tau_j and
// alpha_j = R[j, j] are stored, then flag[j] is raised.  Every CTA applies the
// reflectors in order to the columns it owns.  Look-ahead: the owner of column
// j+1 updates that column with reflector j first and publishes reflector j+1
// before it updates its other columns, so the serial chain per column is one
// column update plus one reflector construction.  Waits are bounded: after
// kSpinLimit polls a CTA records an error and returns.
constexpr long long kSpinLimit = 1LL << 24;

// Block-wide dot of v (shared, rows j..d-1) with column cc (global).
SNS_D double block_dot_col(const double* v, const double* cc, int64_t j, int64_t d, double* red) {
  double s = 0.0;
  for (int64_t i = j + threadIdx.x; i < d; i += blockDim.x) s = fma(v[i], cc[i], s);
  return block_sum(s, red);
}

// Builds reflector j from column j (already updated by reflectors < j):
// scales W[j+1:, j] by 1/v0 in place, stores alpha in W[j, j] and tau in taus[j].
SNS_D void build_reflector(double* W, int64_t d, int64_t j, double* taus, double* red) {
  double* cj = W + j * d;
  double part = 0.0;
  for (int64_t i = j + threadIdx.x; i < d; i += blockDim.x) part = fma(cj[i], cj[i], part);
  const double nrm2 = block_sum(part, red);
  const double x0 = cj[j];
  const double normx = sqrt(nrm2);
  double alpha = x0, tau = 0.0, inv_v0 = 0.0;
  if (normx > 0.0) {
    alpha = (x0 >= 0.0) ? -normx : normx;
    const double v0 = x0 - alpha;
    tau = -v0 / alpha;
    inv_v0 = 1.0 / v0;
  }
  for (int64_t i = j + 1 + threadIdx.x; i < d; i += blockDim.x) cj[i] *= inv_v0;
  __syncthreads();
  if (threadIdx.x == 0) {
    cj[j] = alpha;
    taus[j] = tau;
  }
}

SNS_D void publish(int* flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicExch(flag, 1);
}

// Returns false (and records the error) if the flag never came.
SNS_D bool wait_flag(int* flag, int* err) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const bool got = spin_until_ge(reinterpret_cast<volatile int*>(flag), 1, kSpinLimit);
    if (!got) atomicExch(err, 1);
    __threadfence();
    ok = got ? 1 : 0;
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(kQrThreads)
qr_coop_kernel(double* __restrict__ W, int64_t d, int64_t q, double* __restrict__ taus, int* __restrict__ flags,
               int* __restrict__ err) {
  extern __shared__ double vsm[];   // reflector rows j..d-1
  __shared__ double red[32];
  const int64_t G = gridDim.x, b = blockIdx.x;
  const int64_t steps = q < d ? q : d;
  // reflector 0: built by the owner of column 0 before the loop
  if (b == 0) {
    build_reflector(W, d, 0, taus, red);
    publish(flags + 0);
  }
  for (int64_t j = 0; j < steps; ++j) {
    if (b != j % G) {
      if (!wait_flag(flags + j, err)) return;
    }
    // load v_j and tau_j (through L2: written by another SM)
    const double* cj = W + j * d;
    for (int64_t i = j + threadIdx.x; i < d; i += blockDim.x) vsm[i] = (i == j) ? 1.0 : __ldcg(cj + i);
    __syncthreads();
    const double tau = __ldcg(taus + j);
    // look-ahead column j+1
    const int64_t c1 = j + 1;
    if (c1 < q && c1 % G == b) {
      double* cc = W + c1 * d;
      if (tau != 0.0) {
        const double f = tau * block_dot_col(vsm, cc, j, d, red);
        for (int64_t i = j + threadIdx.x; i < d; i += blockDim.x) cc[i] = fma(-f, vsm[i], cc[i]);
        __syncthreads();
      }
      if (c1 < steps) {
        build_reflector(W, d, c1, taus, red);
        publish(flags + c1);
      }
    }
    // remaining owned columns
    if (tau != 0.0) {
      int64_t c = c1 + 1;
      c += ((b - c) % G + G) % G;               // first owned column > j + 1
      for (; c < q; c += G) {
        double* cc = W + c * d;
        const double f = tau * block_dot_col(vsm, cc, j, d, red);
        for (int64_t i = j + threadIdx.x; i < d; i += blockDim.x) cc[i] = fma(-f, vsm[i], cc[i]);
      }
    }
    __syncthreads();
  }
}

// Rank check + back substitution of a factorised problem on one CTA.
__global__ void __launch_bounds__(kQrThreads) qr_finish_kernel(QrOut o) {
  extern __shared__ double zsm[];
  __shared__ double red[32];
  qr_finish_cta(o.W, o.d, o.q, o.x, o.status, o.sres, zsm, red);
}

int qr_coop_grid(int64_t q) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, qr_coop_kernel, kQrThreads, 0);
  const int64_t cap = (int64_t)num_sms() * std::max(occ, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(q, cap), num_sms()));
}

size_t qr_coop_ws_bytes(int64_t q) { return (size_t)q * 8 + (size_t)q * 4 + 256 + 64; }

sns_status qr_solve_coop(const QrOut& o, void* ws, cudaStream_t st) {
  uint8_t* w = static_cast<uint8_t*>(ws);
  double* taus = reinterpret_cast<double*>(w);
  int* flags = reinterpret_cast<int*>(w + (((size_t)o.q * 8 + 255) & ~(size_t)255));
  int* err = flags + o.q;
  SNS_CUDA_TRY(cudaMemsetAsync(flags, 0, (size_t)o.q * 4 + 4, st));
  const size_t smem = (size_t)o.d * 8;
  SNS_CUDA_TRY(raise_smem_limit((const void*)qr_coop_kernel));
  const int grid = qr_coop_grid(o.q);
  double* W = o.W;
  int64_t d = o.d, q = o.q;
  void* args[] = {&W, &d, &q, &taus, &flags, &err};
  {
    SNS_PROF(K_QR, st);
    SNS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)qr_coop_kernel, dim3(grid), dim3(kQrThreads), args, smem,
                                             st));
  }
  const size_t zs = (size_t)std::max<int64_t>(o.q, 1) * 8;
  SNS_CUDA_TRY(raise_smem_limit((const void*)qr_finish_kernel));
  {
    SNS_PROF(K_QR, st);
    qr_finish_kernel<<<1, kQrThreads, zs, st>>>(o);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

// Explicit R^{-1} (upper triangular, FP64) for the preconditioner applications
// of the iterative phase.  One CTA per column j solves R y = e_j by
// column-oriented back substitution with the running column in shared memory:
// at step k every thread reads y_k = y[k] / R[k, k] (final, since step k only
// updates rows i < k), the owner of row k records it, and all threads update
// their rows i < k; one barrier per step.  Writes Rinv (row-major) and its
// transpose RinvT (row-major).  With `identity`, writes the identity
// (unpreconditioned iteration).
__global__ void __launch_bounds__(256) rinv_kernel(const double* __restrict__ W, int64_t ldw, int64_t n,
                                                   double* __restrict__ Rinv, double* __restrict__ RinvT,
                                                   int identity) {
  extern __shared__ double ycol[];   // n
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) ycol[i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    if (!identity) {
      for (int64_t k = j; k >= 0; --k) {
        const double yk = ycol[k] / W[k * ldw + k];
        const double* rk = W + k * ldw;          // column k of R: rows 0..k
        __syncthreads();                         // everyone has read y[k]
        if (threadIdx.x == 0) ycol[k] = yk;
        for (int64_t i = threadIdx.x; i < k; i += blockDim.x) ycol[i] = fma(-rk[i], yk, ycol[i]);
        __syncthreads();
      }
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = (i <= j) ? ycol[i] : 0.0;
      Rinv[i * n + j] = v;
      RinvT[j * n + i] = v;
    }
    __syncthreads();
  }
}

sns_status rinv_build(const double* W, int64_t ldw, int64_t n, double* Rinv, double* RinvT, bool identity,
                      cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)num_sms() * 4));
  const size_t smem = (size_t)n * 8;
  SNS_CUDA_TRY(raise_smem_limit((const void*)rinv_kernel));
  {
    SNS_PROF(K_RINV, st);
    rinv_kernel<<<grid, 256, smem, st>>>(W, ldw, n, Rinv, RinvT, identity ? 1 : 0);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

}  // namespace sns
