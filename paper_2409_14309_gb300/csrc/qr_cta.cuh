// One-CTA FP64 Householder QR and back substitution of a column-major d x q
// matrix [SA | Sb] (the solve step of sketch-and-solve, Sec. 1.2 step 3), shared
// by the single-problem and the batched kernels.
#pragma once
#include "common.cuh"

namespace sns {

constexpr double kQrU64 = 1.1102230246251565e-16;  // 2^-53

// One CTA factorises one problem held column-major in global memory (L2
// resident at these sizes), then checks the rank and back-substitutes.
SNS_D void qr_factor_cta(double* __restrict__ W, int64_t d, int64_t q, double* v, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int64_t j = 0; j < q && j < d; ++j) {
    double* cj = W + j * d;
    double part = 0.0;
    for (int64_t i = j + tid; i < d; i += nt) {
      const double x = cj[i];
      part = fma(x, x, part);
    }
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
    for (int64_t i = j + tid; i < d; i += nt) v[i] = (i == j) ? 1.0 : cj[i] * inv_v0;
    __syncthreads();
    if (tid == 0) cj[j] = alpha;
    if (tau != 0.0) {
      for (int64_t c = j + 1 + wid; c < q; c += nw) {
        double* cc = W + c * d;
        double s = 0.0;
        for (int64_t i = j + lane; i < d; i += 32) s = fma(v[i], cc[i], s);
        s = warp_sum(s);
        const double f = tau * s;
        for (int64_t i = j + lane; i < d; i += 32) cc[i] = fma(-f, v[i], cc[i]);
      }
    }
    __syncthreads();
  }
}

// Copies 8 bytes global -> shared without staging through registers
// (cp.async; completion per thread via commit/wait groups).
SNS_D void cp_async8(double* dst_smem, const double* src) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(a), "l"(src) : "memory");
}
SNS_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
SNS_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Column-oriented back substitution on one CTA: solves R y = y0 in place for
// rows 0..kend of y (shared memory), where R is upper triangular, column k at
// W + k * ldw, and rd[k] = 1 / R[k, k].  Step k: y_k = y[k] * rd[k] (final,
// since step k writes only rows i < k), then y[i] -= R[i, k] y_k for i < k.
// Each thread owns the rows i = tid (mod blockDim.x), so one barrier per step
// suffices (row k - 1 is read by all only after it).  With RING > 0 the thread
// streams its rows of columns k-1, k-2, ... into a shared-memory ring of RING
// columns (ldr doubles apart) with cp.async, RING - 1 columns ahead, so the
// serial chain never waits on L2.  emit(k, y_k) is called by thread 0.
template <int RING, typename Emit>
SNS_D void tri_backsolve_cta(const double* __restrict__ W, int64_t ldw, int64_t kend, double* y, const double* rd,
                             double* ring, int64_t ldr, Emit emit) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if constexpr (RING > 0) {
    auto issue = [&](int64_t k) {
      if (k >= 0) {
        const double* rk = W + k * ldw;
        double* slot = ring + (k % RING) * ldr;
        for (int64_t i = tid; i < k; i += nt) cp_async8(slot + i, rk + i);
      }
      cp_async_commit();
    };
    for (int p = 0; p < RING - 1; ++p) issue(kend - p);
    for (int64_t k = kend; k >= 0; --k) {
      issue(k - (RING - 1));
      cp_async_wait<RING - 1>();
      const double yk = y[k] * rd[k];
      if (tid == 0) emit(k, yk);
      const double* slot = ring + (k % RING) * ldr;
      for (int64_t i = tid; i < k; i += nt) y[i] = fma(-slot[i], yk, y[i]);
      __syncthreads();
    }
    cp_async_wait<0>();
  } else {
    for (int64_t k = kend; k >= 0; --k) {
      const double yk = y[k] * rd[k];
      if (tid == 0) emit(k, yk);
      const double* rk = W + k * ldw;
      for (int64_t i = tid; i < k; i += nt) y[i] = fma(-rk[i], yk, y[i]);
      __syncthreads();
    }
  }
}

// Rank check and back substitution x = R^{-1} z.  Shared memory `sm` holds
// 2 (q - 1) doubles (z, then the reciprocals of R's diagonal) plus, with
// RING > 0, RING * (q - 1) doubles for the column ring.
template <int RING = 0>
SNS_D void qr_finish_cta(const double* __restrict__ W, int64_t d, int64_t q, double* __restrict__ x,
                         int32_t* status, double* sres, double* sm, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t n = q - 1;
  double mx = 0.0;
  for (int64_t i = tid; i < n; i += nt) mx = fmax(mx, fabs(W[i * d + i]));
  // block max via the sum helper's staging area
  mx = warp_max(mx);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = mx;
  __syncthreads();
  double gmax = 0.0;
  for (int w = 0; w < (nt >> 5); ++w) gmax = fmax(gmax, red[w]);
  __syncthreads();
  int bad = 0;
  for (int64_t i = tid; i < n; i += nt) bad |= (fabs(W[i * d + i]) <= (double)n * kQrU64 * gmax) ? 1 : 0;
  bad = __syncthreads_or(bad);
  if (tid == 0) {
    if (status) *status = (bad || gmax == 0.0) ? SNS_ERANK : SNS_OK;
    if (sres) *sres = (n < d) ? fabs(W[n * d + n]) : 0.0;
  }
  if (!x) return;
  const bool zero = bad || gmax == 0.0;
  double* z = sm;
  double* rd = sm + n;
  for (int64_t i = tid; i < n; i += nt) {
    z[i] = W[n * d + i];
    rd[i] = 1.0 / W[i * d + i];
  }
  __syncthreads();
  tri_backsolve_cta<RING>(W, d, n - 1, z, rd, sm + 2 * n, n, [&](int64_t k, double xk) { x[k] = zero ? 0.0 : xk; });
}

}  // namespace sns
