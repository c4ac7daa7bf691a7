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

// Rank check and back substitution x = R^{-1} z, column-oriented: after x_k is
// known, z[0:k] -= R[0:k, k] x_k.  z lives in shared memory.
SNS_D void qr_finish_cta(const double* __restrict__ W, int64_t d, int64_t q, double* __restrict__ x,
                         int32_t* status, double* sres, double* z, double* red) {
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
  for (int64_t i = tid; i < n; i += nt) z[i] = W[n * d + i];
  __syncthreads();
  for (int64_t k = n - 1; k >= 0; --k) {
    const double xk = z[k] / W[k * d + k];
    __syncthreads();
    if (tid == 0) {
      z[k] = xk;
      x[k] = (bad || gmax == 0.0) ? 0.0 : xk;
    }
    for (int64_t i = tid; i < k; i += nt) z[i] = fma(-W[k * d + i], xk, z[i]);
    __syncthreads();
  }
}


}  // namespace sns
