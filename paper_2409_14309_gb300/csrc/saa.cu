// Sketch-and-apply (SAA-SAS, named beside SAP-SAS in Sec. 2.1 of arXiv
// 2409.14309, after Meier, Nakatsukasa, Townsend & Webb 2023): instead of
// applying R^-1 implicitly in every iteration, the preconditioned matrix
// Y = A R^-1 is formed once, explicitly, and the iteration runs on Y.
//
// On the GPU the refinement structure of the SAP path is kept (residual passes
// on the original A with FP64-class accumulation); only the inner solver
// changes: conjugate gradients on Y^T Y dz = Y^T r = R^-T g with the identity
// as preconditioner (CGLS on Y: the Krylov iterates LSQR on Y also produces),
// whose passes read Y instead of A, then x += R^-1 dz.
//
// Kernels here:
//  * form_y: Y = A R^-1 (m x n, same precision as A; R^-1 is the FP64
//    row-major upper-triangular inverse built from the QR of SA).  A register-
//    tiled SIMT product: a CTA owns 64 (FP32) or 32 (FP64) rows and 256
//    columns; warp w owns 32 of the columns, so the triangular structure of
//    R^-1 (R^-1[k][j] = 0 for k > j) is skipped warp-uniformly.  Products
//    accumulate in the precision of A (FP32 for FP32 input).
//  * tri_matvec: out = M v or out += M v for an n x n FP64 row-major M
//    (R^-T g before a cycle, R^-1 dz after it).
//  * ident_fill: the identity preconditioner.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace sns {

// Tile shape of form_y.  FP32: a thread owns 16 rows x 4 columns; the 32 lanes
// of a warp are 4 row groups x 8 column groups, so a warp covers 64 rows x 32
// columns and the CTA's 8 warps cover 64 rows x 256 columns.  FP64 halves the
// rows per thread (register budget).  K advances in steps of kYK.
constexpr int kYWarps = 8;
constexpr int kYCols = 32 * kYWarps;      // 256 columns per CTA
constexpr int kYK = 16;
template <typename T>
struct YCfg {
  static constexpr int TR = sizeof(T) == 4 ? 16 : 8;   // rows per thread
  static constexpr int BM = 4 * TR;                    // rows per CTA
  static constexpr int LD = BM + 16 / (int)sizeof(T);  // padded row of the transposed A tile (16 bytes)
};

template <typename T>
__global__ void __launch_bounds__(kYWarps * 32)
form_y_kernel(const T* __restrict__ A, int64_t lda, int64_t m, int64_t n, const double* __restrict__ Rinv,
              T* __restrict__ Y, int64_t ldy) {
  constexpr int TR = YCfg<T>::TR, BM = YCfg<T>::BM, LD = YCfg<T>::LD;
  __shared__ __align__(16) T As[kYK][LD];          // A tile, transposed (k-major), rows padded
  __shared__ __align__(16) T Bs[kYK][kYCols];      // R^-1 tile
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int lr = lane >> 3, lc = lane & 7;           // row group 0..3, column group 0..7
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t col0 = (int64_t)blockIdx.y * kYCols;
  const int64_t wcol0 = col0 + 32 * w;               // this warp's first column
  const int64_t kend = std::min<int64_t>(n, col0 + kYCols);   // R^-1[k][j] = 0 for k > j
  T acc[TR][4];
#pragma unroll
  for (int r = 0; r < TR; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = T(0);

  for (int64_t k0 = 0; k0 < kend; k0 += kYK) {
    // A tile: BM rows x kYK columns; consecutive threads read consecutive k of a row
    for (int e = tid; e < BM * kYK; e += kYWarps * 32) {
      const int r = e / kYK, kk = e % kYK;
      const int64_t gi = row0 + r, gk = k0 + kk;
      As[kk][r] = (gi < m && gk < n) ? __ldg(A + gi * lda + gk) : T(0);
    }
    // R^-1 tile: kYK rows x 256 columns, rounded to T
    for (int e = tid; e < kYK * kYCols; e += kYWarps * 32) {
      const int kk = e / kYCols, c = e % kYCols;
      const int64_t gk = k0 + kk, gj = col0 + c;
      Bs[kk][c] = (gk < n && gj < n && gk <= gj) ? (T)__ldg(Rinv + gk * n + gj) : T(0);
    }
    __syncthreads();
    if (k0 <= wcol0 + 31) {                          // warp-uniform: this k-tile meets the warp's columns
#pragma unroll
      for (int kk = 0; kk < kYK; ++kk) {
        T a[TR], bv[4];
#pragma unroll
        for (int r = 0; r < TR; ++r) a[r] = As[kk][lr * TR + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][32 * w + lc * 4 + c];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fma(a[r], bv[c], acc[r][c]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < TR; ++r) {
    const int64_t gi = row0 + lr * TR + r;
    if (gi >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t gj = wcol0 + lc * 4 + c;
      if (gj < n) Y[gi * ldy + gj] = acc[r][c];
    }
  }
}

// out = M v (ACCUM: out += M v), M n x n FP64 row-major; one warp per row.
template <bool ACCUM>
__global__ void __launch_bounds__(128)
tri_matvec_kernel(const double* __restrict__ M, int64_t n, const double* __restrict__ v, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n; i += nw) {
    const double* mr = M + i * n;
    double acc = 0.0;
    for (int64_t k = lane; k < n; k += 32) acc = fma(__ldg(mr + k), v[k], acc);
    acc = warp_sum(acc);
    if (lane == 0) out[i] = ACCUM ? out[i] + acc : acc;
  }
}

__global__ void ident_fill_kernel(double* __restrict__ P, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
    P[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// ---------------------------------------------------------------------------
int64_t saa_ldy(int64_t n, bool f64) { return f64 ? n : (n + 3) / 4 * 4; }
size_t saa_y_bytes(int64_t m, int64_t n, bool f64) { return (size_t)m * saa_ldy(n, f64) * (f64 ? 8 : 4); }

template <typename T>
static sns_status launch_form_y(const T* A, int64_t lda, int64_t m, int64_t n, const double* Rinv, T* Y,
                                int64_t ldy, cudaStream_t st) {
  const dim3 grid((unsigned)((m + YCfg<T>::BM - 1) / YCfg<T>::BM), (unsigned)((n + kYCols - 1) / kYCols));
  {
    SNS_PROF(K_SAA_Y, st);
    form_y_kernel<T><<<grid, kYWarps * 32, 0, st>>>(A, lda, m, n, Rinv, Y, ldy);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

sns_status saa_form_y(const DenseArgs& a, const double* Rinv, void* Y, cudaStream_t st, int64_t ldy) {
  if (ldy <= 0) ldy = saa_ldy(a.n, a.f64);
  if (a.f64)
    return launch_form_y<double>(static_cast<const double*>(a.A), a.lda, a.m, a.n, Rinv, static_cast<double*>(Y),
                                 ldy, st);
  return launch_form_y<float>(static_cast<const float*>(a.A), a.lda, a.m, a.n, Rinv, static_cast<float*>(Y), ldy,
                              st);
}

sns_status saa_matvec(const double* M, int64_t n, const double* v, double* out, bool accumulate, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, (n + 3) / 4);
  {
    SNS_PROF(K_MATVEC, st);
    if (accumulate) tri_matvec_kernel<true><<<grid, 128, 0, st>>>(M, n, v, out);
    else tri_matvec_kernel<false><<<grid, 128, 0, st>>>(M, n, v, out);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

sns_status ident_build(double* P, int64_t n, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n * n + 255) / 256, 1024));
  {
    SNS_PROF(K_RINV, st);
    ident_fill_kernel<<<grid, 256, 0, st>>>(P, n);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

}  // namespace sns
