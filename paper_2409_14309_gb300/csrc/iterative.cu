// Sketch-and-precondition (SAP-SAS, Sec. 2.1 of arXiv 2409.14309, after Meier
// et al. 2023): R from the QR of SA right-preconditions an iterative solve on
// the original A, started from the sketch-and-solve answer x^.
//
// Precision layout: passes over A run on the FP32 pipes.  A pure FP32 Krylov
// iteration on an A with condition number ~1e6 stalls near eta ~ 1e-4 (the
// FP32 products perturb A by ~u32 ||A||, which moves the solution by
// kappa^2 u32 ||r|| / ||A||).  Accuracy is therefore won back by iterative
// refinement: each outer step computes g = A^T (b - A x) with compensated
// ("FP64-class") accumulation, then an inner conjugate-gradient solve of the
// R-preconditioned normal equations  (R^-T A^T A R^-1) y = R^-T g  with FP32
// passes (CGLS: the Krylov iterates LSQR also produces in exact arithmetic),
// and x += R^-1 y.  The inner solve only needs a relative accuracy < 1 per
// outer step, so its FP32 error does not limit the final accuracy.
//
// Kernels:
//  * resid_pass: one read of A and b: r_i = b_i - a_i.x, g += a_i r_i, ||r||^2,
//    and (first time) ||A||_F^2.  Dense FP32 uses error-free transformations
//    (TwoProdFMA + TwoSum, the Dot2 scheme of Ogita, Rump & Oishi 2005);
//    FP64 input and CSR use FP64 arithmetic.
//  * normal_pass: one read of A: w = A^T (A z) with z = R^-1 p in FP32.
//  * small FP64 kernels for R^-1 / R^-T applications and the CG recurrences.
// Both passes leave per-CTA partial vectors; the last CTA to finish (ticket)
// adds them in CTA order in FP64, so results are deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace sns {

constexpr int kPassThreads = 256;
constexpr int kPassWarps = kPassThreads / 32;
constexpr int kPassU = 2;       // rows in flight per warp

int iter_grid() { return num_sms() * 2; }

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t iter_ws_bytes(int64_t n, int grid) {
  size_t s = 0;
  s += 2 * al256((size_t)n * n * 8);          // Rinv, RinvT
  s += 9 * al256((size_t)n * 8);              // g w rhs y res p qv z
  s += al256(64 * 8);                         // scal
  s += 3 * al256((size_t)n * 4);              // xhi xlo z32
  s += al256((size_t)grid * n * 4);           // part
  s += al256((size_t)grid * (n + 4) * 8);     // partd
  s += al256(64);                             // ticket
  return s;
}

IterWs iter_ws_carve(void* base, int64_t n, int grid) {
  IterWs W{};
  uint8_t* p = static_cast<uint8_t*>(base);
  auto take = [&](size_t b) { uint8_t* r = p; p += al256(b); return r; };
  W.Rinv = (double*)take((size_t)n * n * 8);
  W.RinvT = (double*)take((size_t)n * n * 8);
  W.g = (double*)take(n * 8);
  W.w = (double*)take(n * 8);
  W.rhs = (double*)take(n * 8);
  W.y = (double*)take(n * 8);
  W.res = (double*)take(n * 8);
  W.p = (double*)take(n * 8);
  W.qv = (double*)take(n * 8);
  W.z = (double*)take(n * 8);
  (void)take(n * 8);
  W.scal = (double*)take(64 * 8);
  W.xhi = (float*)take(n * 4);
  W.xlo = (float*)take(n * 4);
  W.z32 = (float*)take(n * 4);
  W.part = (float*)take((size_t)grid * n * 4);
  W.partd = (double*)take((size_t)grid * (n + 4) * 8);
  W.ticket = (uint32_t*)take(64);
  W.grid = grid;
  return W;
}

// Scalar slots in W.scal.
enum { kRR = 0, kRnorm2 = 1, kAnorm2 = 2, kEta = 3, kGnorm2 = 4, kRnorm = 5, kPQ = 6 };

// Last-CTA detection: returns true in every thread of the CTA that finished last.
SNS_D bool last_cta(uint32_t* ticket) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// ------------------------------------------------------------------ dense FP32
// Compensated accumulator: value = hi + lo, lo collecting rounding errors.
struct Comp {
  float hi, lo;
};
SNS_D void comp_fma(Comp& c, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  const float s = c.hi + p;
  const float bb = s - c.hi;
  const float e = (c.hi - (s - bb)) + (p - bb);
  c.hi = s;
  c.lo += pe + e;
}
SNS_D void comp_add(Comp& c, float p) {
  const float s = c.hi + p;
  const float bb = s - c.hi;
  const float e = (c.hi - (s - bb)) + (p - bb);
  c.hi = s;
  c.lo += e;
}

template <int VEC>
SNS_D void ldv(const float* p, float (&v)[VEC]) {
  if constexpr (VEC == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    v[0] = __ldg(p);
  }
}

template <int VEC, int NCH>
__global__ void __launch_bounds__(kPassThreads)
resid_pass_f32(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n,
               const double* __restrict__ x, double* __restrict__ partd, uint32_t* __restrict__ ticket,
               double* __restrict__ g, double* __restrict__ scal, int want_anorm) {
  __shared__ double sred[kPassWarps][3];
  extern __shared__ __align__(16) double dsm[];      // [kPassWarps][n] doubles
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float xh[NCH][VEC], xl[NCH][VEC];
  bool ok[NCH];
  Comp gacc[NCH][VEC];
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int64_t c0 = (int64_t)q * 32 * VEC + lane * VEC;
    ok[q] = c0 < n;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const double xv = (c0 + v < n) ? x[c0 + v] : 0.0;
      xh[q][v] = (float)xv;
      xl[q][v] = (float)(xv - (double)xh[q][v]);
      gacc[q][v] = {0.f, 0.f};
    }
  }
  double rr = 0.0;
  float an = 0.f;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = gw * kPassU; r0 < m; r0 += nw * kPassU) {
    float a[kPassU][NCH][VEC];
    float bv[kPassU];
#pragma unroll
    for (int u = 0; u < kPassU; ++u) {
      const bool rok = r0 + u < m;
      const float* rp = A + (r0 + u) * lda + lane * VEC;
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        if (rok && ok[q]) ldv<VEC>(rp + q * 32 * VEC, a[u][q]);
        else
#pragma unroll
          for (int v = 0; v < VEC; ++v) a[u][q][v] = 0.f;
      }
      bv[u] = rok ? __ldg(b + r0 + u) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPassU; ++u) {
      Comp s = {0.f, 0.f};
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          comp_fma(s, a[u][q][v], xh[q][v]);
          s.lo = fmaf(a[u][q][v], xl[q][v], s.lo);
          an = fmaf(a[u][q][v], a[u][q][v], an);
        }
      // warp sum of the compensated dot
      float hi = s.hi, lo = s.lo;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        Comp c = {hi, lo + ol};
        comp_add(c, oh);
        hi = c.hi;
        lo = c.lo;
      }
      // r = b - dot (as hi + lo)
      Comp r = {bv[u], 0.f};
      comp_add(r, -hi);
      r.lo -= lo;
      const float rh = r.hi + r.lo;
      const float rl = r.lo - (rh - r.hi);
      if (lane == 0 && r0 + u < m) rr = fma((double)rh + rl, (double)rh + rl, rr);
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          comp_fma(gacc[q][v], a[u][q][v], rh);
          gacc[q][v].lo = fmaf(a[u][q][v], rl, gacc[q][v].lo);
        }
    }
  }
  // CTA reduction in FP64, fixed order
  double* myrow = dsm + (size_t)w * n;
#pragma unroll
  for (int q = 0; q < NCH; ++q)
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int64_t c = (int64_t)q * 32 * VEC + lane * VEC + v;
      if (c < n) myrow[c] = (double)gacc[q][v].hi + (double)gacc[q][v].lo;
    }
  const double rrw = warp_sum(rr);
  const double anw = warp_sum((double)an);
  if (lane == 0) { sred[w][0] = rrw; sred[w][1] = anw; }
  __syncthreads();
  double* out = partd + (size_t)blockIdx.x * (n + 4);
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    double s = 0.0;
    for (int ww = 0; ww < kPassWarps; ++ww) s += dsm[(size_t)ww * n + c];
    out[c] = s;
  }
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int ww = 0; ww < kPassWarps; ++ww) { a0 += sred[ww][0]; a1 += sred[ww][1]; }
    out[n] = a0;
    out[n + 1] = a1;
  }
  if (last_cta(ticket)) {
    for (int64_t c = threadIdx.x; c < n + 2; c += blockDim.x) {
      double s = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) s += __ldcg(partd + (size_t)k * (n + 4) + c);
      if (c < n) g[c] = s;
      else if (c == n) scal[kRnorm2] = s;
      else if (want_anorm) scal[kAnorm2] = s;
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

template <int VEC, int NCH>
__global__ void __launch_bounds__(kPassThreads)
normal_pass_f32(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ z32,
                float* __restrict__ part, uint32_t* __restrict__ ticket, double* __restrict__ wout) {
  extern __shared__ __align__(16) float fsm[];       // [kPassWarps][n]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float zr[NCH][VEC], acc[NCH][VEC];
  bool ok[NCH];
#pragma unroll
  for (int q = 0; q < NCH; ++q) {
    const int64_t c0 = (int64_t)q * 32 * VEC + lane * VEC;
    ok[q] = c0 < n;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      zr[q][v] = (c0 + v < n) ? z32[c0 + v] : 0.f;
      acc[q][v] = 0.f;
    }
  }
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = gw * kPassU; r0 < m; r0 += nw * kPassU) {
    float a[kPassU][NCH][VEC];
#pragma unroll
    for (int u = 0; u < kPassU; ++u) {
      const bool rok = r0 + u < m;
      const float* rp = A + (r0 + u) * lda + lane * VEC;
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        if (rok && ok[q]) ldv<VEC>(rp + q * 32 * VEC, a[u][q]);
        else
#pragma unroll
          for (int v = 0; v < VEC; ++v) a[u][q][v] = 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < kPassU; ++u) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) t = fmaf(a[u][q][v], zr[q][v], t);
      t = warp_sum(t);
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[q][v] = fmaf(t, a[u][q][v], acc[q][v]);
    }
  }
  float* myrow = fsm + (size_t)w * n;
#pragma unroll
  for (int q = 0; q < NCH; ++q)
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int64_t c = (int64_t)q * 32 * VEC + lane * VEC + v;
      if (c < n) myrow[c] = acc[q][v];
    }
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * n;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    float s = 0.f;
    for (int ww = 0; ww < kPassWarps; ++ww) s += fsm[(size_t)ww * n + c];
    out[c] = s;
  }
  if (last_cta(ticket)) {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      double s = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) s += (double)__ldcg(part + (size_t)k * n + c);
      wout[c] = s;
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// ------------------------------------------------------------------ FP64 dense
__global__ void __launch_bounds__(kPassThreads)
resid_pass_f64(const double* __restrict__ A, int64_t lda, const double* __restrict__ b, int64_t m, int64_t n,
               const double* __restrict__ x, double* __restrict__ partd, uint32_t* __restrict__ ticket,
               double* __restrict__ g, double* __restrict__ scal, int want_anorm) {
  extern __shared__ __align__(16) double dsm[];      // x[n], gl[n]
  double* xs = dsm;
  double* gl = dsm + n;
  __shared__ double sred[kPassWarps][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) { xs[c] = x[c]; gl[c] = 0.0; }
  __syncthreads();
  double rr = 0.0, an = 0.0;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < m; r += nw) {
    const double* rp = A + r * lda;
    double s = 0.0;
    for (int64_t c = lane; c < n; c += 32) { const double a = rp[c]; s = fma(a, xs[c], s); an = fma(a, a, an); }
    s = warp_sum(s);
    const double rv = b[r] - s;
    if (lane == 0) rr = fma(rv, rv, rr);
    for (int64_t c = lane; c < n; c += 32) atomicAdd(gl + c, rp[c] * rv);
  }
  rr = warp_sum(rr);
  an = warp_sum(an);
  if (lane == 0) { sred[w][0] = rr; sred[w][1] = an; }
  __syncthreads();
  double* out = partd + (size_t)blockIdx.x * (n + 4);
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) out[c] = gl[c];
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int ww = 0; ww < kPassWarps; ++ww) { a0 += sred[ww][0]; a1 += sred[ww][1]; }
    out[n] = a0;
    out[n + 1] = a1;
  }
  if (last_cta(ticket)) {
    for (int64_t c = threadIdx.x; c < n + 2; c += blockDim.x) {
      double s = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) s += __ldcg(partd + (size_t)k * (n + 4) + c);
      if (c < n) g[c] = s;
      else if (c == n) scal[kRnorm2] = s;
      else if (want_anorm) scal[kAnorm2] = s;
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

__global__ void __launch_bounds__(kPassThreads)
normal_pass_f64(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n, const double* __restrict__ z,
                double* __restrict__ partd, uint32_t* __restrict__ ticket, double* __restrict__ wout) {
  extern __shared__ __align__(16) double dsm[];      // z[n], wl[n]
  double* zs = dsm;
  double* wl = dsm + n;
  const int lane = threadIdx.x & 31;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) { zs[c] = z[c]; wl[c] = 0.0; }
  __syncthreads();
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = gw; r < m; r += nw) {
    const double* rp = A + r * lda;
    double s = 0.0;
    for (int64_t c = lane; c < n; c += 32) s = fma(rp[c], zs[c], s);
    s = warp_sum(s);
    for (int64_t c = lane; c < n; c += 32) atomicAdd(wl + c, rp[c] * s);
  }
  __syncthreads();
  double* out = partd + (size_t)blockIdx.x * (n + 4);
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) out[c] = wl[c];
  if (last_cta(ticket)) {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      double s = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) s += __ldcg(partd + (size_t)k * (n + 4) + c);
      wout[c] = s;
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// ------------------------------------------------------------------ CSR
__global__ void __launch_bounds__(kPassThreads)
resid_pass_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
               const float* __restrict__ b, int64_t m, int64_t n, const double* __restrict__ x,
               double* __restrict__ partd, uint32_t* __restrict__ ticket, double* __restrict__ g,
               double* __restrict__ scal, int want_anorm) {
  extern __shared__ __align__(16) double dsm[];      // x[n], gl[n]
  double* xs = dsm;
  double* gl = dsm + n;
  __shared__ double sred[kPassWarps][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) { xs[c] = x[c]; gl[c] = 0.0; }
  __syncthreads();
  double rr = 0.0, an = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = rowptr[r], e1 = rowptr[r + 1];
    double s = 0.0;
    for (int64_t e = e0; e < e1; ++e) {
      const uint32_t c = (uint32_t)col[e];
      const double a = val[e];
      if (c < (uint64_t)n) s = fma(a, xs[c], s);
      an = fma(a, a, an);
    }
    const double rv = (double)b[r] - s;
    rr = fma(rv, rv, rr);
    for (int64_t e = e0; e < e1; ++e) {
      const uint32_t c = (uint32_t)col[e];
      if (c < (uint64_t)n) atomicAdd(gl + c, (double)val[e] * rv);
    }
  }
  rr = warp_sum(rr);
  an = warp_sum(an);
  if (lane == 0) { sred[w][0] = rr; sred[w][1] = an; }
  __syncthreads();
  double* out = partd + (size_t)blockIdx.x * (n + 4);
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) out[c] = gl[c];
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int ww = 0; ww < kPassWarps; ++ww) { a0 += sred[ww][0]; a1 += sred[ww][1]; }
    out[n] = a0;
    out[n + 1] = a1;
  }
  if (last_cta(ticket)) {
    for (int64_t c = threadIdx.x; c < n + 2; c += blockDim.x) {
      double s = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) s += __ldcg(partd + (size_t)k * (n + 4) + c);
      if (c < n) g[c] = s;
      else if (c == n) scal[kRnorm2] = s;
      else if (want_anorm) scal[kAnorm2] = s;
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

__global__ void __launch_bounds__(kPassThreads)
normal_pass_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
                int64_t m, int64_t n, const float* __restrict__ z32, float* __restrict__ part,
                uint32_t* __restrict__ ticket, double* __restrict__ wout) {
  extern __shared__ __align__(16) float fsm[];       // z[n], wl[n]
  float* zs = fsm;
  float* wl = fsm + n;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) { zs[c] = z32[c]; wl[c] = 0.f; }
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = rowptr[r], e1 = rowptr[r + 1];
    float s = 0.f;
    for (int64_t e = e0; e < e1; ++e) {
      const uint32_t c = (uint32_t)col[e];
      if (c < (uint64_t)n) s = fmaf(val[e], zs[c], s);
    }
    for (int64_t e = e0; e < e1; ++e) {
      const uint32_t c = (uint32_t)col[e];
      if (c < (uint64_t)n) atomicAdd(wl + c, val[e] * s);
    }
  }
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * n;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) out[c] = wl[c];
  if (last_cta(ticket)) {
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      double s = 0.0;
      for (unsigned k = 0; k < gridDim.x; ++k) s += (double)__ldcg(part + (size_t)k * n + c);
      wout[c] = s;
    }
    if (threadIdx.x == 0) *ticket = 0;
  }
}

// ------------------------------------------------------------------ launchers
template <int VEC, int NCH>
static sns_status launch_dense_f32(const DenseArgs& a, const IterWs& W, const double* x, bool resid, bool want_anorm,
                                   cudaStream_t st) {
  const float* A = static_cast<const float*>(a.A);
  if (resid) {
    const size_t smem = (size_t)kPassWarps * a.n * 8;
    auto k = resid_pass_f32<VEC, NCH>;
    SNS_CUDA_TRY(raise_smem_limit((const void*)k));
    {
      SNS_PROF(K_RESID, st);
    k<<<W.grid, kPassThreads, smem, st>>>(A, a.lda, static_cast<const float*>(a.b), a.m, a.n, x, W.partd, W.ticket,
                                          W.g, W.scal, want_anorm ? 1 : 0);
    }
  } else {
    const size_t smem = (size_t)kPassWarps * a.n * 4;
    auto k = normal_pass_f32<VEC, NCH>;
    SNS_CUDA_TRY(raise_smem_limit((const void*)k));
    {
      SNS_PROF(K_NORMAL, st);
    k<<<W.grid, kPassThreads, smem, st>>>(A, a.lda, a.m, a.n, W.z32, W.part, W.ticket, W.w);
    }
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

static sns_status dense_f32_dispatch(const DenseArgs& a, const IterWs& W, const double* x, bool resid,
                                     bool want_anorm, cudaStream_t st) {
  const bool v4 = (a.lda % 4 == 0) && (a.n % 4 == 0) && ((uintptr_t)a.A % 16 == 0);
  if (v4) {
    if (a.n <= 128) return launch_dense_f32<4, 1>(a, W, x, resid, want_anorm, st);
    if (a.n <= 256) return launch_dense_f32<4, 2>(a, W, x, resid, want_anorm, st);
    if (a.n <= 512) return launch_dense_f32<4, 4>(a, W, x, resid, want_anorm, st);
    if (a.n <= 1024) return launch_dense_f32<4, 8>(a, W, x, resid, want_anorm, st);
  } else {
    if (a.n <= 32) return launch_dense_f32<1, 1>(a, W, x, resid, want_anorm, st);
    if (a.n <= 128) return launch_dense_f32<1, 4>(a, W, x, resid, want_anorm, st);
    if (a.n <= 256) return launch_dense_f32<1, 8>(a, W, x, resid, want_anorm, st);
    if (a.n <= 512) return launch_dense_f32<1, 16>(a, W, x, resid, want_anorm, st);
    if (a.n <= 1024) return launch_dense_f32<1, 32>(a, W, x, resid, want_anorm, st);
  }
  return SNS_EINVAL;
}

sns_status resid_pass(const DenseArgs* da, const CsrArgs* ca, const double* x, const IterWs& W, bool want_anorm,
                      cudaStream_t st) {
  if (da && !da->f64) return dense_f32_dispatch(*da, W, x, true, want_anorm, st);
  if (da) {
    const size_t smem = (size_t)da->n * 16;
    SNS_CUDA_TRY(raise_smem_limit((const void*)resid_pass_f64));
    {
      SNS_PROF(K_RESID, st);
    resid_pass_f64<<<W.grid, kPassThreads, smem, st>>>(static_cast<const double*>(da->A), da->lda,
                                                       static_cast<const double*>(da->b), da->m, da->n, x, W.partd,
                                                       W.ticket, W.g, W.scal, want_anorm ? 1 : 0);
    }
  } else {
    const size_t smem = (size_t)ca->n * 16;
    SNS_CUDA_TRY(raise_smem_limit((const void*)resid_pass_csr));
    {
      SNS_PROF(K_RESID, st);
    resid_pass_csr<<<W.grid, kPassThreads, smem, st>>>(ca->rowptr, ca->col, ca->val, ca->b, ca->m, ca->n, x, W.partd,
                                                       W.ticket, W.g, W.scal, want_anorm ? 1 : 0);
    }
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

sns_status normal_pass(const DenseArgs* da, const CsrArgs* ca, const IterWs& W, cudaStream_t st) {
  if (da && !da->f64) return dense_f32_dispatch(*da, W, nullptr, false, false, st);
  if (da) {
    const size_t smem = (size_t)da->n * 16;
    SNS_CUDA_TRY(raise_smem_limit((const void*)normal_pass_f64));
    {
      SNS_PROF(K_NORMAL, st);
    normal_pass_f64<<<W.grid, kPassThreads, smem, st>>>(static_cast<const double*>(da->A), da->lda, da->m, da->n,
                                                        W.z, W.partd, W.ticket, W.w);
    }
  } else {
    const size_t smem = (size_t)ca->n * 8;
    SNS_CUDA_TRY(raise_smem_limit((const void*)normal_pass_csr));
    {
      SNS_PROF(K_NORMAL, st);
    normal_pass_csr<<<W.grid, kPassThreads, smem, st>>>(ca->rowptr, ca->col, ca->val, ca->m, ca->n, W.z32, W.part,
                                                        W.ticket, W.w);
    }
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

// out_i = sum_k M[i, k] v[k] (row-major n x n); optional FP32 copy and
// accum += alpha * out.  One warp per row.
__global__ void small_matvec_kernel(const double* __restrict__ M, const double* __restrict__ v, int64_t n,
                                    double* __restrict__ out, float* __restrict__ out32, double alpha,
                                    double* __restrict__ accum) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n; i += nw) {
    double s = 0.0;
    for (int64_t k = lane; k < n; k += 32) s = fma(M[i * n + k], v[k], s);
    s = warp_sum(s);
    if (lane == 0) {
      if (out) out[i] = s;
      if (out32) out32[i] = (float)s;
      if (accum) accum[i] += alpha * s;
    }
  }
}

sns_status small_matvec(const double* M, const double* v, int64_t n, double* out, float* out32, double alpha,
                        double* accum, cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)num_sms()));
  {
    SNS_PROF(K_MATVEC, st);
  small_matvec_kernel<<<grid, 256, 0, st>>>(M, v, n, out, out32, alpha, accum);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

// CG on (R^-T A^T A R^-1) y = rhs.  init: y = 0, res = p = rhs, rr = |res|^2.
__global__ void cg_init_kernel(const double* __restrict__ rhs, int64_t n, double* y, double* res, double* p,
                               double* scal) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = rhs[i];
    y[i] = 0.0;
    res[i] = r;
    p[i] = r;
    s = fma(r, r, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) scal[kRR] = s;
}
// step: q = R^-T w (given in qv); alpha = rr / (p.q); y += alpha p;
// res -= alpha q; rr' = |res|^2; p = res + (rr'/rr) p.
__global__ void cg_step_kernel(int64_t n, const double* __restrict__ qv, double* y, double* res, double* p,
                               double* scal) {
  __shared__ double red[32];
  double pq = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) pq = fma(p[i], qv[i], pq);
  pq = block_sum(pq, red);
  const double rr = scal[kRR];
  const double alpha = (pq > 0.0 && rr > 0.0) ? rr / pq : 0.0;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    y[i] = fma(alpha, p[i], y[i]);
    const double r = fma(-alpha, qv[i], res[i]);
    res[i] = r;
    s = fma(r, r, s);
  }
  const double rr2 = block_sum(s, red);
  const double beta = (rr > 0.0) ? rr2 / rr : 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = fma(beta, p[i], res[i]);
  __syncthreads();
  if (threadIdx.x == 0) scal[kRR] = rr2;
}

sns_status cg_init(const IterWs& W, int64_t n, cudaStream_t st) {
  {
    SNS_PROF(K_CG, st);
  cg_init_kernel<<<1, 512, 0, st>>>(W.rhs, n, W.y, W.res, W.p, W.scal);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}
sns_status cg_step(const IterWs& W, int64_t n, cudaStream_t st) {
  {
    SNS_PROF(K_CG, st);
  cg_step_kernel<<<1, 512, 0, st>>>(n, W.qv, W.y, W.res, W.p, W.scal);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

// eta = ||g|| / (||A||_F ||r||) after a resid_pass; copies
// [eta, ||r||, ||g||, ||A||_F] to host_out (pinned) asynchronously.
__global__ void eta_kernel(const double* __restrict__ g, int64_t n, double* scal) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(g[i], g[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double rn = sqrt(scal[kRnorm2]);
    const double an = sqrt(scal[kAnorm2]);
    const double gn = sqrt(s);
    scal[kGnorm2] = s;
    scal[kRnorm] = rn;
    scal[kEta] = (rn > 0.0 && an > 0.0) ? gn / (an * rn) : 0.0;
    scal[8] = scal[kEta];
    scal[9] = rn;
    scal[10] = gn;
    scal[11] = an;
  }
}
sns_status eta_eval(const IterWs& W, int64_t n, double* host_out, cudaStream_t st) {
  {
    SNS_PROF(K_ETA, st);
  eta_kernel<<<1, 512, 0, st>>>(W.g, n, W.scal);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  SNS_CUDA_TRY(cudaMemcpyAsync(host_out, W.scal + 8, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  return SNS_OK;
}

}  // namespace sns
