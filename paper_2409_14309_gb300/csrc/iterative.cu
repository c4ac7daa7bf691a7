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

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace sns {

constexpr int kPassThreads = 256;
constexpr int kPassWarps = kPassThreads / 32;
constexpr int kNormU = 4;       // rows in flight per warp (normal pass)

int iter_grid() { return num_sms() * 4; }

// Grid of one full wave for a pass kernel: SMs x resident CTAs per SM (capped
// by the workspace's partial rows).  A second, partial wave would stream the
// end of A at a fraction of the occupancy.  Cached per (device, kernel, smem).
static int pass_grid(const void* fn, size_t smem, int cap) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, fn, smem);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return std::min(it->second, cap);
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kPassThreads, smem) != cudaSuccess || occ < 1) occ = 1;
  const int g = num_sms() * occ;
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = g;
  return std::min(g, cap);
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t iter_ws_bytes(int64_t n, int grid) {
  size_t s = 0;
  s += 3 * al256((size_t)n * n * 8);          // Rinv, RinvT, P
  s += 6 * al256((size_t)n * 8);              // g w z rx s dx
  s += al256(64 * 8);                         // scal
  s += 3 * al256((size_t)n * 4);              // xhi xlo z32
  s += al256((size_t)grid * n * 4);           // part
  s += al256((size_t)grid * (n + 4) * 8);     // partd
  s += al256(64 * 4);                         // tickets (groups + top)
  s += al256((size_t)64 * (n + 4) * 8);       // level-2 partials
  return s;
}

IterWs iter_ws_carve(void* base, int64_t n, int grid) {
  IterWs W{};
  uint8_t* p = static_cast<uint8_t*>(base);
  auto take = [&](size_t b) { uint8_t* r = p; p += al256(b); return r; };
  W.Rinv = (double*)take((size_t)n * n * 8);
  W.RinvT = (double*)take((size_t)n * n * 8);
  W.P = (double*)take((size_t)n * n * 8);
  W.g = (double*)take(n * 8);
  W.w = (double*)take(n * 8);
  W.z = (double*)take(n * 8);
  W.rx = (double*)take(n * 8);
  W.s = (double*)take(n * 8);
  W.dx = (double*)take(n * 8);
  W.scal = (double*)take(64 * 8);
  W.xhi = (float*)take(n * 4);
  W.xlo = (float*)take(n * 4);
  W.z32 = (float*)take(n * 4);
  W.part = (float*)take((size_t)grid * n * 4);
  W.partd = (double*)take((size_t)grid * (n + 4) * 8);
  W.ticket = (uint32_t*)take(64 * 4);
  W.lvl2 = (double*)take((size_t)64 * (n + 4) * 8);
  W.grid = grid;
  return W;
}

// Scalar slots in W.scal.
enum { kRR = 0, kRnorm2 = 1, kAnorm2 = 2, kEta = 3, kGnorm2 = 4, kRnorm = 5, kPQ = 6 };
// Inner-loop control (device-side, so the host never waits inside a cycle):
// kStop2 = the CG residual^2 at which the cycle ends, kDone = nonzero once it
// has (later launches of the cycle return at once), kPasses = normal passes run.
enum { kStop2 = 16, kDone = 17, kPasses = 18 };
// Slots 8..12 are copied to the host after each residual pass:
// eta, ||r||, ||g||, ||A||_F, passes run.
constexpr int kHostSlots = 5;
// Per-cycle floor of the CG residual reduction: the FP32 passes (z = R^-1 p
// rounded to FP32 and A z in FP32) limit what one refinement cycle can gain,
// and iterating past that only repeats work the next cycle redoes.
constexpr double kInnerFloor = 4e-3;

// Deterministic two-level reduction of per-CTA partial rows.  CTA b has
// written its row part[b * stride + c], c < nc.  CTAs form groups of 32; the
// last CTA of a group (ticket) adds the group's rows in CTA order (FP64) into
// lvl2[group]; the last group to finish adds the group sums in group order and
// calls emit(c, value).  Tickets are reset by the CTAs that consume them.
// Returns true in the one CTA that emitted (after a barrier, so its emitted
// values are visible to all its threads).
constexpr int kRedGroup = 32;
// Sum of the cnt values p[k * stride] in the order k = 0, 1, ...; loads are
// issued in batches (32 floats: a group of float partials in one L2 round
// trip; 8 doubles, which keeps the FP64 passes' register budget).
template <typename PT>
SNS_D double sum_strided(const PT* __restrict__ p, int64_t stride, int64_t cnt) {
  constexpr int K = sizeof(PT) == 4 ? 32 : 8;
  double acc = 0.0;
  for (int64_t k0 = 0; k0 < cnt; k0 += K) {
    PT v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = (k0 + k < cnt) ? __ldcg(p + (k0 + k) * stride) : PT(0);
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k0 + k < cnt) acc += (double)v[k];
  }
  return acc;
}
template <typename PT, typename F>
SNS_D bool tree_reduce(const PT* __restrict__ part, int64_t stride, int64_t nc, uint32_t* __restrict__ tickets,
                       double* __restrict__ lvl2, F&& emit) {
  __shared__ int s_last;
  const int64_t G = gridDim.x;
  const int64_t ngroups = (G + kRedGroup - 1) / kRedGroup;
  const int64_t grp = blockIdx.x / kRedGroup;
  const int64_t gsize = min((int64_t)kRedGroup, G - grp * kRedGroup);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(tickets + grp, 1u) == (uint32_t)(gsize - 1));
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int64_t c = threadIdx.x; c < nc; c += blockDim.x)
    lvl2[grp * stride + c] = sum_strided(part + grp * kRedGroup * stride + c, stride, gsize);
  if (threadIdx.x == 0) tickets[grp] = 0;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(tickets + ngroups, 1u) == (uint32_t)(ngroups - 1));
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int64_t c = threadIdx.x; c < nc; c += blockDim.x) emit(c, sum_strided(lvl2 + c, stride, ngroups));
  if (threadIdx.x == 0) tickets[ngroups] = 0;
  __syncthreads();
  return true;
}

// Vectors of the inner solver (see pcg_alpha), passed by value to the kernels.
struct PcgVecs {
  double *z, *rx, *s, *dx, *w, *scal;
  float* z32;
};
static PcgVecs pcg_vecs(const IterWs& W) { return PcgVecs{W.z, W.rx, W.s, W.dx, W.w, W.scal, W.z32}; }
constexpr int kPcgTicket = 63;           // ticket slot of pcg_matvec (tree_reduce uses 0..ngroups)

// One-CTA reductions for the O(n) epilogues: warp sums, then thread 0 adds
// the per-warp partials in order (the FP64 pipe is narrow, so no thread
// repeats work another has done).  Result valid in thread 0 only.
SNS_D double cta_sum0(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// ---------------------------------------------------------------------------
// Inner solver: preconditioned CG on the normal equations A^T A dx = g with
// M^-1 = P = R^-1 R^-T, R from the QR of SA (Sec. 1.2, sketch-and-precondition).
// In exact arithmetic this is CG on R^-T A^T A R^-1 y = R^-T g with dx = R^-1 y,
// written in x-space so one iteration needs one pass over A (w = A^T A z) and
// one n x n matvec (s = P r); all O(n) work runs in the final CTA of those two
// kernels:
//   pass epilogue:   alpha = rr / (z.w);  dx += alpha z;  r -= alpha w
//   matvec epilogue: rr' = r.s;  beta = rr'/rr;  z = s + beta z (and FP32 z)
// P is formed once per solve; kappa(P) = kappa(R)^2 costs ~kappa(R)^2 eps64
// relative accuracy in P r, irrelevant for a preconditioner.
SNS_D void pcg_alpha(const PcgVecs& V, int64_t n) {
  __shared__ double red[32];
  __shared__ double s_alpha;
  double zw = 0.0;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) zw = fma(V.z[c], V.w[c], zw);
  zw = cta_sum0(zw, red);
  if (threadIdx.x == 0) {
    const double rr = V.scal[kRR];
    s_alpha = (zw > 0.0 && rr > 0.0) ? rr / zw : 0.0;
  }
  __syncthreads();
  const double alpha = s_alpha;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    V.dx[c] = fma(alpha, V.z[c], V.dx[c]);
    V.rx[c] = fma(-alpha, V.w[c], V.rx[c]);
  }
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

SNS_D Comp comp_plus(Comp a, Comp b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return {s, (a.lo + b.lo) + e};
}
SNS_D Comp comp_shfl_xor(Comp c, int o) {
  return {__shfl_xor_sync(0xffffffffu, c.hi, o), __shfl_xor_sync(0xffffffffu, c.lo, o)};
}

// Residual pass, dense FP32: r = b - A x in FP64-class accuracy, g = A^T r,
// ||r||^2 (and ||A||_F^2 when ANORM).  Each warp takes U rows (4 or 2) at a time.
// Row dots use exact products (TwoProdFMA) and compensated sums, since b - A x
// cancels; a U-row reduce-scatter butterfly leaves row u's total in lanes
// u*32/U .. (u+1)*32/U - 1.  For g, EXACT adds every product exactly (TwoProdFMA,
// compensated sum, plus the a * r_lo term).  Without EXACT, per column the U
// rows' products a * r_hi are summed in FP32 and that partial is added with a
// compensated sum: the accumulation stays error-free to float-float accuracy
// and only per-term rounding remains, so ||dg|| <~ eps32 * max_i ||a_i|| * ||r||,
// i.e. an eta floor of at most ~3e-8 even when one row carries all of ||A||_F
// (below 1e-9 for incoherent rows at m >= 1e4).
template <int VEC, int NCH, int U, bool ANORM, bool EXACT>
__global__ void __launch_bounds__(kPassThreads)
resid_pass_f32(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n,
               const double* __restrict__ x, double* __restrict__ partd, uint32_t* __restrict__ ticket, double* __restrict__ lvl2,
               double* __restrict__ g, double* __restrict__ scal) {
  static_assert(U == 4 || U == 2, "reduce-scatter over 4 or 2 rows");
  constexpr int kLpr = 32 / U;                        // lanes per row after the butterfly
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
  const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
  const int urow = lane / kLpr;                       // row of the lane group after the butterfly
  // ||r||^2 of the rows this lane group finishes (the group's first lane counts)
  Comp rrc = {0.f, 0.f};
  float an = 0.f;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = gw * U; r0 < m; r0 += nw * U) {
    float a[U][NCH][VEC];
    float bv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
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
    Comp s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      s[u] = {0.f, 0.f};
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          comp_fma(s[u], a[u][q][v], xh[q][v]);
          s[u].lo = fmaf(a[u][q][v], xl[q][v], s[u].lo);
          if (ANORM) an = fmaf(a[u][q][v], a[u][q][v], an);
        }
    }
    // reduce-scatter: xor 16 splits rows {0,1} | {2,3}, xor 8 splits the pair,
    // xor 4, 2, 1 finish the row's sum
    Comp kk;
    float bme;
    if constexpr (U == 4) {
      Comp k0 = up16 ? s[2] : s[0], k1 = up16 ? s[3] : s[1];
      const Comp g0 = up16 ? s[0] : s[2], g1 = up16 ? s[1] : s[3];
      k0 = comp_plus(k0, comp_shfl_xor(g0, 16));
      k1 = comp_plus(k1, comp_shfl_xor(g1, 16));
      kk = up8 ? k1 : k0;
      kk = comp_plus(kk, comp_shfl_xor(up8 ? k0 : k1, 8));
      bme = urow == 0 ? bv[0] : urow == 1 ? bv[1] : urow == 2 ? bv[2] : bv[3];
    } else {
      kk = up16 ? s[1] : s[0];
      kk = comp_plus(kk, comp_shfl_xor(up16 ? s[0] : s[1], 16));
      kk = comp_plus(kk, comp_shfl_xor(kk, 8));
      bme = up16 ? bv[1] : bv[0];
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) kk = comp_plus(kk, comp_shfl_xor(kk, o));
    // r = b - dot for this lane's row
    Comp r = {bme, 0.f};
    comp_add(r, -kk.hi);
    r.lo -= kk.lo;
    const float rh = r.hi + r.lo;
    const float rl = r.lo - (rh - r.hi);
    if (lane % kLpr == 0 && r0 + urow < m) {
      comp_fma(rrc, rh, rh);
      rrc.lo = fmaf(2.f * rh, rl, rrc.lo);
    }
    float rhu[U];
#pragma unroll
    for (int u = 0; u < U; ++u) rhu[u] = __shfl_sync(0xffffffffu, rh, kLpr * u);
    if constexpr (EXACT) {
      float rlu[U];
#pragma unroll
      for (int u = 0; u < U; ++u) rlu[u] = __shfl_sync(0xffffffffu, rl, kLpr * u);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int q = 0; q < NCH; ++q)
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            comp_fma(gacc[q][v], a[u][q][v], rhu[u]);
            gacc[q][v].lo = fmaf(a[u][q][v], rlu[u], gacc[q][v].lo);
          }
    } else {
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          float t = a[0][q][v] * rhu[0];
#pragma unroll
          for (int u = 1; u < U; ++u) t = fmaf(a[u][q][v], rhu[u], t);
          comp_add(gacc[q][v], t);
        }
    }
  }
  // CTA reduction in float-float (fixed order), one conversion to FP64 per
  // column: FP64 instructions are scarce on this part
  float2* myrow = reinterpret_cast<float2*>(dsm) + (size_t)w * n;
#pragma unroll
  for (int q = 0; q < NCH; ++q)
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const int64_t c = (int64_t)q * 32 * VEC + lane * VEC + v;
      if (c < n) myrow[c] = make_float2(gacc[q][v].hi, gacc[q][v].lo);
    }
  const double rrw = warp_sum(lane % kLpr == 0 ? (double)rrc.hi + (double)rrc.lo : 0.0);
  const double anw = ANORM ? warp_sum((double)an) : 0.0;
  if (lane == 0) { sred[w][0] = rrw; sred[w][1] = anw; }
  __syncthreads();
  double* out = partd + (size_t)blockIdx.x * (n + 4);
  const float2* rows = reinterpret_cast<const float2*>(dsm);
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    const float2 f0 = rows[c];
    Comp acc = {f0.x, f0.y};
#pragma unroll
    for (int ww = 1; ww < kPassWarps; ++ww) {
      const float2 f = rows[(size_t)ww * n + c];
      acc = comp_plus(acc, Comp{f.x, f.y});
    }
    out[c] = (double)acc.hi + (double)acc.lo;
  }
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int ww = 0; ww < kPassWarps; ++ww) { a0 += sred[ww][0]; a1 += sred[ww][1]; }
    out[n] = a0;
    out[n + 1] = a1;
  }
  tree_reduce(partd, n + 4, n + 2, ticket, lvl2, [&](int64_t c, double s) {
    if (c < n) g[c] = s;
    else if (c == n) scal[kRnorm2] = s;
    else if (ANORM) scal[kAnorm2] = s;
  });
}

template <int VEC, int NCH>
__global__ void __launch_bounds__(kPassThreads)
normal_pass_f32(const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, const float* __restrict__ z32,
                float* __restrict__ part, uint32_t* __restrict__ ticket, double* __restrict__ lvl2, PcgVecs V) {
  extern __shared__ __align__(16) float fsm[];       // [kPassWarps][n]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // A is read-only: start this warp's first rows towards L2 before waiting
  // for the kernel that produced z
  {
    const int64_t pc = min((int64_t)lane * ((n + 31) / 32), n - 1);   // lanes spread over the row
#pragma unroll
    for (int u = 0; u < kNormU; ++u)
      if (gw * kNormU + u < m) prefetch_l2(A + (gw * kNormU + u) * lda + pc);
  }
  grid_dep_wait();
  if (V.scal[kDone] != 0.0) return;                  // this refinement cycle has already converged
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
  for (int64_t r0 = gw * kNormU; r0 < m; r0 += nw * kNormU) {
    float a[kNormU][NCH][VEC];
#pragma unroll
    for (int u = 0; u < kNormU; ++u) {
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
    for (int u = 0; u < kNormU; ++u) {
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
  grid_dep_trigger();                                // the next kernel may start launching
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
  if (tree_reduce(part, n, n, ticket, lvl2, [&](int64_t c, double s) { V.w[c] = s; })) pcg_alpha(V, n);
}

// ------------------------------------------------------------------ FP64 dense
__global__ void __launch_bounds__(kPassThreads)
resid_pass_f64(const double* __restrict__ A, int64_t lda, const double* __restrict__ b, int64_t m, int64_t n,
               const double* __restrict__ x, double* __restrict__ partd, uint32_t* __restrict__ ticket, double* __restrict__ lvl2,
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
  tree_reduce(partd, n + 4, n + 2, ticket, lvl2, [&](int64_t c, double s) {
    if (c < n) g[c] = s;
    else if (c == n) scal[kRnorm2] = s;
    else if (want_anorm) scal[kAnorm2] = s;
  });
}

__global__ void __launch_bounds__(kPassThreads)
normal_pass_f64(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n, const double* __restrict__ z,
                double* __restrict__ partd, uint32_t* __restrict__ ticket, double* __restrict__ lvl2, PcgVecs V) {
  grid_dep_wait();
  if (V.scal[kDone] != 0.0) return;
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
  if (tree_reduce(partd, n + 4, n, ticket, lvl2, [&](int64_t c, double s) { V.w[c] = s; })) pcg_alpha(V, n);
}

// ------------------------------------------------------------------ CSR
// ------------------------------------------------------------------ CSR
// Rows are walked in chunks of 32 per warp (chunks go round the CTAs first, so
// neighbouring chunks land on different SMs).  A row with at most kLongRow
// nonzeros belongs to one lane, which loads its entries kRowBatch at a time.
// Longer rows (dense rows) are taken by whole warps with coalesced loads: from
// a per-CTA queue drained after the main loop (default), or right after the
// chunk's short rows (DET).  Products are scattered into a per-warp
// accumulator row (PERWARP; else one per CTA when n is too large) with shared
// atomics (default).  With DET (asked for, and PERWARP) the
// passes are bitwise reproducible: the walk is warp-uniform and static (every
// row is taken by the same warp every run), lanes of one scatter step that hit
// the same column add in lane order (rank rounds, plain shared stores),
// accumulator rows are added in warp order and reduced across CTAs with
// tree_reduce.  The rank rounds cost ~3.8x per pass (measured), hence opt-in.
constexpr int kLongRow = 32;
constexpr int kRowBatch = 8;             // entries loaded at once per lane (short rows)
constexpr int kLongBatch = 16;           // per lane for long rows: 512-entry rows in one round trip
// Shared memory up to which the CSR passes keep one accumulator row per warp.
constexpr size_t kCsrSmemPerWarpMax = 100 * 1024;

// The widest per-warp layout is the exact residual pass: x (double) plus one
// double row per warp.
int64_t csr_det_max_n() { return (int64_t)(kCsrSmemPerWarpMax / (8 + (size_t)kPassWarps * 8)); }


constexpr int kLongQueue = 256;          // long rows queued per CTA (more are done in place)
struct LongQueue {
  int64_t row[kLongQueue];
  int count, next;
};

// Walks this warp's chunks (default passes); short rows go to
// short_row(row, e0, e1) on their lane; long rows are queued for the CTA (or
// passed to long_row(row, e0, e1) by the whole warp when the queue is full),
// and all warps of the CTA drain the queue after the main loop, one long row
// per warp at a time (balances the dense rows across the CTA's warps).
template <typename Short, typename Long>
SNS_D void csr_walk_queued(const int64_t* __restrict__ rowptr, int64_t m, LongQueue& Q, Short&& short_row,
                           Long&& long_row) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)w * gridDim.x + blockIdx.x;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (threadIdx.x == 0) {
    Q.count = 0;
    Q.next = 0;
  }
  __syncthreads();
  for (int64_t r0 = gw * 32; r0 < m; r0 += nw * 32) {
    const int64_t r = r0 + lane;
    int64_t e0 = 0, e1 = 0;
    if (r < m) {
      e0 = __ldg(rowptr + r);
      e1 = __ldg(rowptr + r + 1);
    }
    const bool lng = (e1 - e0) > kLongRow;
    if (!lng && r < m) short_row(r, e0, e1);
    bool inline_long = false;
    if (lng) {
      const int slot = atomicAdd(&Q.count, 1);
      if (slot < kLongQueue) Q.row[slot] = r;
      else inline_long = true;
    }
    unsigned lm = __ballot_sync(0xffffffffu, inline_long);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      long_row(r0 + src, __shfl_sync(0xffffffffu, e0, src), __shfl_sync(0xffffffffu, e1, src));
    }
  }
  __syncthreads();
  const int nq = min(Q.count, kLongQueue);
  for (;;) {
    int k = 0;
    if (lane == 0) k = atomicAdd(&Q.next, 1);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= nq) break;
    const int64_t row = Q.row[k];
    long_row(row, __ldg(rowptr + row), __ldg(rowptr + row + 1));
  }
}

// Walks this warp's chunks (reproducible passes); short rows go to
// short_row(row, e0, e1, active), called by the whole warp with `active` set on
// the lanes that own a short row; the chunk's long rows then go to
// long_row(row, e0, e1), each taken by the whole warp, in lane order (no queue
// shared by the CTA's warps, whose slot order would vary from run to run).
template <typename Short, typename Long>
SNS_D void csr_walk_static(const int64_t* __restrict__ rowptr, int64_t m, Short&& short_row, Long&& long_row) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)w * gridDim.x + blockIdx.x;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = gw * 32; r0 < m; r0 += nw * 32) {
    const int64_t r = r0 + lane;
    int64_t e0 = 0, e1 = 0;
    if (r < m) {
      e0 = __ldg(rowptr + r);
      e1 = __ldg(rowptr + r + 1);
    }
    const bool lng = (e1 - e0) > kLongRow;
    short_row(r < m ? r : 0, e0, e1, !lng && r < m);
    unsigned lm = __ballot_sync(0xffffffffu, lng);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      long_row(r0 + src, __shfl_sync(0xffffffffu, e0, src), __shfl_sync(0xffffffffu, e1, src));
    }
  }
}

// One scatter step of a warp into its accumulator row acc: lane l adds v at
// column c (c outside [0, n) adds nothing).  DET (a per-warp accumulator):
// lanes with equal c add in lane order, one plain shared read-modify-write per
// round; otherwise shared atomics (equal-address lanes apply in an order that
// may vary, and the accumulator may be shared by the CTA's warps).
template <bool DET, typename T>
SNS_D void warp_scatter(T* acc, int64_t n, int32_t c, T v) {
  const bool ok = (uint32_t)c < (uint64_t)n;
  if constexpr (DET) {
    const int lane = threadIdx.x & 31;
    const int32_t key = ok ? c : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const unsigned rank = ok ? (unsigned)__popc(peers & ((1u << lane) - 1u)) : 0u;
    const unsigned rounds = __reduce_max_sync(0xffffffffu, rank) + 1u;
    for (unsigned rr = 0; rr < rounds; ++rr) {
      if (ok && rank == rr) acc[c] += v;
      __syncwarp();
    }
  } else {
    if (ok) atomicAdd(acc + c, v);
  }
}

template <bool PERWARP, bool DET>
__global__ void __launch_bounds__(kPassThreads, 3)
normal_pass_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
                int64_t m, int64_t n, const float* __restrict__ z32, float* __restrict__ part,
                uint32_t* __restrict__ ticket, double* __restrict__ lvl2, PcgVecs V) {
  extern __shared__ __align__(16) float fsm[];       // z[n], accumulators [PERWARP ? warps : 1][n]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int nacc = PERWARP ? kPassWarps : 1;
  grid_dep_wait();
  if (V.scal[kDone] != 0.0) return;
  float* zs = fsm;
  float* acc = fsm + n;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) zs[c] = z32[c];
  for (int64_t c = threadIdx.x; c < nacc * n; c += blockDim.x) acc[c] = 0.f;
  __syncthreads();
  float* wl = acc + (PERWARP ? (size_t)w * n : 0);
  // default: one lane per short row, shared atomics
  auto short_row = [&](int64_t, int64_t e0, int64_t e1) {
    int32_t cc[kRowBatch];
    float vv[kRowBatch];
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u) {
      const bool ok = e0 + u < e1;
      cc[u] = ok ? __ldg(col + e0 + u) : -1;
      vv[u] = ok ? __ldg(val + e0 + u) : 0.f;
    }
    float t = 0.f;
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u)
      if ((uint32_t)cc[u] < (uint64_t)n) t = fmaf(vv[u], zs[cc[u]], t);
    if (e0 + kRowBatch >= e1) {                        // the usual case: one batch holds the row
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u)
        if ((uint32_t)cc[u] < (uint64_t)n) atomicAdd(wl + cc[u], vv[u] * t);
      return;
    }
    // rows of 9..32 entries: finish the dot, then scatter from the top
    for (int64_t e = e0 + kRowBatch; e < e1; ++e) {
      const uint32_t c = (uint32_t)__ldg(col + e);
      if (c < (uint64_t)n) t = fmaf(__ldg(val + e), zs[c], t);
    }
    for (int64_t e = e0; e < e1; ++e) {
      const uint32_t c = (uint32_t)__ldg(col + e);
      if (c < (uint64_t)n) atomicAdd(wl + c, __ldg(val + e) * t);
    }
  };
  // DET: the whole warp steps through its short rows together (rank rounds)
  auto short_row_det = [&](int64_t, int64_t e0, int64_t e1, bool active) {
    // first batch of the row (all a row has in the usual case)
    int32_t cc[kRowBatch];
    float vv[kRowBatch];
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u) {
      const bool ok = active && e0 + u < e1;
      cc[u] = ok ? __ldg(col + e0 + u) : -1;
      vv[u] = ok ? __ldg(val + e0 + u) : 0.f;
    }
    float t = 0.f;
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u)
      if ((uint32_t)cc[u] < (uint64_t)n) t = fmaf(vv[u], zs[cc[u]], t);
    if (active)                                         // rows of 9..32 entries: finish the dot
      for (int64_t e = e0 + kRowBatch; e < e1; ++e) {
        const uint32_t c = (uint32_t)__ldg(col + e);
        if (c < (uint64_t)n) t = fmaf(__ldg(val + e), zs[c], t);
      }
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u) warp_scatter<PERWARP && DET>(wl, n, cc[u], vv[u] * t);
    for (int64_t eb = e0 + kRowBatch; __any_sync(0xffffffffu, active && eb < e1); eb += kRowBatch) {
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u) {
        const bool ok = active && eb + u < e1;
        cc[u] = ok ? __ldg(col + eb + u) : -1;
        vv[u] = ok ? __ldg(val + eb + u) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u) warp_scatter<PERWARP && DET>(wl, n, cc[u], vv[u] * t);
    }
  };
  auto long_row = [&](int64_t, int64_t a0, int64_t a1) {
    float t = 0.f;
    for (int64_t eb = a0; eb < a1; eb += 32 * kLongBatch) {
      int32_t cc[kLongBatch];
      float vv[kLongBatch];
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u) {
        const int64_t e = eb + u * 32 + lane;
        cc[u] = e < a1 ? __ldg(col + e) : -1;
        vv[u] = e < a1 ? __ldg(val + e) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u)
        if ((uint32_t)cc[u] < (uint64_t)n) t = fmaf(vv[u], zs[cc[u]], t);
    }
    t = warp_sum(t);
    for (int64_t eb = a0; eb < a1; eb += 32 * kLongBatch) {
      int32_t cc[kLongBatch];
      float vv[kLongBatch];
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u) {
        const int64_t e = eb + u * 32 + lane;
        cc[u] = e < a1 ? __ldg(col + e) : -1;
        vv[u] = e < a1 ? __ldg(val + e) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u) warp_scatter<PERWARP && DET>(wl, n, cc[u], vv[u] * t);
    }
  };
  if constexpr (DET) {
    csr_walk_static(rowptr, m, short_row_det, long_row);
  } else {
    __shared__ LongQueue Q;
    csr_walk_queued(rowptr, m, Q, short_row, long_row);
  }
  grid_dep_trigger();
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * n;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < nacc; ++k) t += acc[(size_t)k * n + c];
    out[c] = t;
  }
  if (tree_reduce(part, n, n, ticket, lvl2, [&](int64_t c, double v) { V.w[c] = v; })) pcg_alpha(V, n);
}

// Residual pass on CSR: r_i = b_i - a_i . x with exact products and
// compensated sums (x = x_hi + x_lo in FP32), one FP64 value per row; g = A^T r
// with FP64 shared atomics of a * r (EXACT) or FP32 atomics of a * r_hi.
template <bool EXACT, bool ANORM, bool PERWARP, bool DET>
__global__ void __launch_bounds__(kPassThreads, 2)
resid_pass_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
               const float* __restrict__ b, int64_t m, int64_t n, const double* __restrict__ x,
               double* __restrict__ partd, uint32_t* __restrict__ ticket, double* __restrict__ lvl2, double* __restrict__ g,
               double* __restrict__ scal) {
  using AccT = typename std::conditional<EXACT, double, float>::type;
  extern __shared__ __align__(16) double dsm[];      // x_hi[n], x_lo[n] (FP32), accumulators
  __shared__ double sred[kPassWarps][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int nacc = PERWARP ? kPassWarps : 1;
  float* xh = reinterpret_cast<float*>(dsm);
  float* xl = xh + n;
  AccT* acc = reinterpret_cast<AccT*>(dsm + n);
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    const double xv = x[c];
    xh[c] = (float)xv;
    xl[c] = (float)(xv - (double)xh[c]);
  }
  for (int64_t c = threadIdx.x; c < nacc * n; c += blockDim.x) acc[c] = AccT(0);
  __syncthreads();
  AccT* gl = acc + (PERWARP ? (size_t)w * n : 0);
  Comp rrc = {0.f, 0.f};
  float an = 0.f;
  auto add_entry = [&](Comp& sdot, int32_t c, float a) {
    if ((uint32_t)c < (uint64_t)n) {
      comp_fma(sdot, a, xh[c]);
      sdot.lo = fmaf(a, xl[c], sdot.lo);
    }
    if (ANORM) an = fmaf(a, a, an);
  };
  auto resid_of = [&](float bv, Comp sdot, float& rh, float& rl) {
    Comp rc = {bv, 0.f};
    comp_add(rc, -sdot.hi);
    rc.lo -= sdot.lo;
    rh = rc.hi + rc.lo;
    rl = rc.lo - (rh - rc.hi);
  };
  // one scatter step of the warp: lane adds a * r at column c (c < 0: nothing)
  auto scatter = [&](int32_t c, float a, float rh, double rd) {
    if constexpr (EXACT) warp_scatter<PERWARP && DET, double>(gl, n, c, (double)a * rd);
    else warp_scatter<PERWARP && DET, float>(gl, n, c, a * rh);
  };
  // default: one lane per short row, shared atomics
  auto short_row = [&](int64_t r, int64_t e0, int64_t e1) {
    const float bv = __ldg(b + r);
    int32_t cc[kRowBatch];
    float vv[kRowBatch];
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u) {
      const bool ok = e0 + u < e1;
      cc[u] = ok ? __ldg(col + e0 + u) : -1;
      vv[u] = ok ? __ldg(val + e0 + u) : 0.f;
    }
    Comp sdot = {0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u)
      if (cc[u] >= 0) add_entry(sdot, cc[u], vv[u]);
    for (int64_t e = e0 + kRowBatch; e < e1; ++e) add_entry(sdot, __ldg(col + e), __ldg(val + e));
    float rh, rl;
    resid_of(bv, sdot, rh, rl);
    comp_fma(rrc, rh, rh);
    rrc.lo = fmaf(2.f * rh, rl, rrc.lo);
    const double rd = EXACT ? (double)rh + (double)rl : 0.0;
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u)
      if (cc[u] >= 0) scatter(cc[u], vv[u], rh, rd);
    for (int64_t e = e0 + kRowBatch; e < e1; ++e) scatter(__ldg(col + e), __ldg(val + e), rh, rd);
  };
  // DET: the whole warp steps through its short rows together (rank rounds)
  auto short_row_det = [&](int64_t r, int64_t e0, int64_t e1, bool active) {
    const float bv = active ? __ldg(b + r) : 0.f;
    int32_t cc[kRowBatch];
    float vv[kRowBatch];
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u) {
      const bool ok = active && e0 + u < e1;
      cc[u] = ok ? __ldg(col + e0 + u) : -1;
      vv[u] = ok ? __ldg(val + e0 + u) : 0.f;
    }
    Comp sdot = {0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u)
      if (cc[u] >= 0) add_entry(sdot, cc[u], vv[u]);
    if (active)
      for (int64_t e = e0 + kRowBatch; e < e1; ++e) add_entry(sdot, __ldg(col + e), __ldg(val + e));
    float rh = 0.f, rl = 0.f;
    if (active) {
      resid_of(bv, sdot, rh, rl);
      comp_fma(rrc, rh, rh);
      rrc.lo = fmaf(2.f * rh, rl, rrc.lo);
    }
    const double rd = EXACT ? (double)rh + (double)rl : 0.0;
#pragma unroll
    for (int u = 0; u < kRowBatch; ++u) scatter(cc[u], vv[u], rh, rd);
    for (int64_t eb = e0 + kRowBatch; __any_sync(0xffffffffu, active && eb < e1); eb += kRowBatch) {
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u) {
        const bool ok = active && eb + u < e1;
        cc[u] = ok ? __ldg(col + eb + u) : -1;
        vv[u] = ok ? __ldg(val + eb + u) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kRowBatch; ++u) scatter(cc[u], vv[u], rh, rd);
    }
  };
  auto long_row = [&](int64_t r, int64_t a0, int64_t a1) {
    Comp sdot = {0.f, 0.f};
    for (int64_t eb = a0; eb < a1; eb += 32 * kLongBatch) {
      int32_t cc[kLongBatch];
      float vv[kLongBatch];
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u) {
        const int64_t e = eb + u * 32 + lane;
        cc[u] = e < a1 ? __ldg(col + e) : -1;
        vv[u] = e < a1 ? __ldg(val + e) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u)
        if (cc[u] >= 0) add_entry(sdot, cc[u], vv[u]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sdot = comp_plus(sdot, comp_shfl_xor(sdot, o));
    float rh, rl;
    resid_of(__ldg(b + r), sdot, rh, rl);
    if (lane == 0) {
      comp_fma(rrc, rh, rh);
      rrc.lo = fmaf(2.f * rh, rl, rrc.lo);
    }
    const double rd = EXACT ? (double)rh + (double)rl : 0.0;
    for (int64_t eb = a0; eb < a1; eb += 32 * kLongBatch) {
      int32_t cc[kLongBatch];
      float vv[kLongBatch];
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u) {
        const int64_t e = eb + u * 32 + lane;
        cc[u] = e < a1 ? __ldg(col + e) : -1;
        vv[u] = e < a1 ? __ldg(val + e) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kLongBatch; ++u) scatter(cc[u], vv[u], rh, rd);
    }
  };
  if constexpr (DET) {
    csr_walk_static(rowptr, m, short_row_det, long_row);
  } else {
    __shared__ LongQueue Q;
    csr_walk_queued(rowptr, m, Q, short_row, long_row);
  }
  const double rrw = warp_sum((double)rrc.hi + (double)rrc.lo);
  const double anw = ANORM ? warp_sum((double)an) : 0.0;
  if (lane == 0) {
    sred[w][0] = rrw;
    sred[w][1] = anw;
  }
  __syncthreads();
  double* out = partd + (size_t)blockIdx.x * (n + 4);
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < nacc; ++k) t += (double)acc[(size_t)k * n + c];
    out[c] = t;
  }
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int ww = 0; ww < kPassWarps; ++ww) {
      a0 += sred[ww][0];
      a1 += sred[ww][1];
    }
    out[n] = a0;
    out[n + 1] = a1;
  }
  tree_reduce(partd, n + 4, n + 2, ticket, lvl2, [&](int64_t c, double v) {
    if (c < n) g[c] = v;
    else if (c == n) scal[kRnorm2] = v;
    else if (ANORM) scal[kAnorm2] = v;
  });
}

// ------------------------------------------------------------------ launchers
template <int VEC, int NCH>
static sns_status launch_dense_f32(const DenseArgs& a, const IterWs& W, const double* x, bool resid, bool want_anorm,
                                   bool exact_g, cudaStream_t st) {
  const float* A = static_cast<const float*>(a.A);
  if (resid) {
    const size_t smem = (size_t)kPassWarps * a.n * 8;
    constexpr int U = (VEC * NCH <= 8) ? 4 : 2;      // rows per warp step within the register budget
    auto k = want_anorm ? (exact_g ? resid_pass_f32<VEC, NCH, U, true, true> : resid_pass_f32<VEC, NCH, U, true, false>)
                        : (exact_g ? resid_pass_f32<VEC, NCH, U, false, true> : resid_pass_f32<VEC, NCH, U, false, false>);
    SNS_CUDA_TRY(raise_smem_limit((const void*)k));
    const int grid = pass_grid((const void*)k, smem, W.grid);
    {
      SNS_PROF(K_RESID, st);
    k<<<grid, kPassThreads, smem, st>>>(A, a.lda, static_cast<const float*>(a.b), a.m, a.n, x, W.partd, W.ticket, W.lvl2,
                                        W.g, W.scal);
    }
  } else {
    const size_t smem = (size_t)kPassWarps * a.n * 4;
    auto k = normal_pass_f32<VEC, NCH>;
    SNS_CUDA_TRY(raise_smem_limit((const void*)k));
    const int grid = pass_grid((const void*)k, smem, W.grid);
    {
      SNS_PROF(K_NORMAL, st);
    SNS_CUDA_TRY(launch_dependent(k, dim3(grid), dim3(kPassThreads), smem, st, A, a.lda, a.m, a.n, W.z32, W.part,
                                  W.ticket, W.lvl2, pcg_vecs(W)));
    }
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

static sns_status dense_f32_dispatch(const DenseArgs& a, const IterWs& W, const double* x, bool resid,
                                     bool want_anorm, bool exact_g, cudaStream_t st) {
  const bool v4 = (a.lda % 4 == 0) && (a.n % 4 == 0) && ((uintptr_t)a.A % 16 == 0);
  if (v4) {
    if (a.n <= 128) return launch_dense_f32<4, 1>(a, W, x, resid, want_anorm, exact_g, st);
    if (a.n <= 256) return launch_dense_f32<4, 2>(a, W, x, resid, want_anorm, exact_g, st);
    if (a.n <= 512) return launch_dense_f32<4, 4>(a, W, x, resid, want_anorm, exact_g, st);
    if (a.n <= 1024) return launch_dense_f32<4, 8>(a, W, x, resid, want_anorm, exact_g, st);
  } else {
    if (a.n <= 32) return launch_dense_f32<1, 1>(a, W, x, resid, want_anorm, exact_g, st);
    if (a.n <= 128) return launch_dense_f32<1, 4>(a, W, x, resid, want_anorm, exact_g, st);
    if (a.n <= 256) return launch_dense_f32<1, 8>(a, W, x, resid, want_anorm, exact_g, st);
    if (a.n <= 512) return launch_dense_f32<1, 16>(a, W, x, resid, want_anorm, exact_g, st);
    if (a.n <= 1024) return launch_dense_f32<1, 32>(a, W, x, resid, want_anorm, exact_g, st);
  }
  return SNS_EINVAL;
}

sns_status resid_pass(const DenseArgs* da, const CsrArgs* ca, const double* x, const IterWs& W, bool want_anorm, bool exact_g,
                      cudaStream_t st) {
  if (da && !da->f64) return dense_f32_dispatch(*da, W, x, true, want_anorm, exact_g, st);
  if (da) {
    const size_t smem = (size_t)da->n * 16;
    SNS_CUDA_TRY(raise_smem_limit((const void*)resid_pass_f64));
    {
      SNS_PROF(K_RESID, st);
    resid_pass_f64<<<W.grid, kPassThreads, smem, st>>>(static_cast<const double*>(da->A), da->lda,
                                                       static_cast<const double*>(da->b), da->m, da->n, x, W.partd,
                                                       W.ticket, W.lvl2, W.g, W.scal, want_anorm ? 1 : 0);
    }
  } else {
    const int64_t n = ca->n;
    const size_t esz = exact_g ? 8 : 4;
    const bool perwarp = (size_t)n * 8 + (size_t)kPassWarps * n * esz <= kCsrSmemPerWarpMax;
    const size_t smem = (size_t)n * 8 + (perwarp ? (size_t)kPassWarps : 1) * n * esz;
#define SNS_RCSR(E, A, P) (const void*)resid_pass_csr<E, A, P, false>, (const void*)resid_pass_csr<E, A, P, true>
    const void* fns[2][2][2][2] = {{{{SNS_RCSR(false, false, false)}, {SNS_RCSR(false, false, true)}},
                                    {{SNS_RCSR(false, true, false)}, {SNS_RCSR(false, true, true)}}},
                                   {{{SNS_RCSR(true, false, false)}, {SNS_RCSR(true, false, true)}},
                                    {{SNS_RCSR(true, true, false)}, {SNS_RCSR(true, true, true)}}}};
#undef SNS_RCSR
    const void* fn = fns[exact_g][want_anorm][perwarp][perwarp && ca->det];
    SNS_CUDA_TRY(raise_smem_limit(fn));
    const int grid = pass_grid(fn, smem, W.grid);
    const float* bb = ca->b;
    const double* xx = x;
    void* args[] = {(void*)&ca->rowptr, (void*)&ca->col, (void*)&ca->val, (void*)&bb, (void*)&ca->m, (void*)&ca->n,
                    (void*)&xx, (void*)&W.partd, (void*)&W.ticket, (void*)&W.lvl2, (void*)&W.g, (void*)&W.scal};
    {
      SNS_PROF(K_RESID, st);
      SNS_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kPassThreads), args, smem, st));
    }
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

sns_status normal_pass(const DenseArgs* da, const CsrArgs* ca, const IterWs& W, cudaStream_t st) {
  if (da && !da->f64) return dense_f32_dispatch(*da, W, nullptr, false, false, false, st);
  if (da) {
    const size_t smem = (size_t)da->n * 16;
    SNS_CUDA_TRY(raise_smem_limit((const void*)normal_pass_f64));
    {
      SNS_PROF(K_NORMAL, st);
    normal_pass_f64<<<W.grid, kPassThreads, smem, st>>>(static_cast<const double*>(da->A), da->lda, da->m, da->n,
                                                        W.z, W.partd, W.ticket, W.lvl2, pcg_vecs(W));
    }
  } else {
    const int64_t n = ca->n;
    const bool perwarp = (size_t)(1 + kPassWarps) * n * 4 <= kCsrSmemPerWarpMax;
    const size_t smem = (size_t)(1 + (perwarp ? kPassWarps : 1)) * n * 4;
    auto k = perwarp ? (ca->det ? normal_pass_csr<true, true> : normal_pass_csr<true, false>)
                     : normal_pass_csr<false, false>;
    SNS_CUDA_TRY(raise_smem_limit((const void*)k));
    const int grid = pass_grid((const void*)k, smem, W.grid);
    {
      SNS_PROF(K_NORMAL, st);
      SNS_CUDA_TRY(launch_dependent(k, dim3(grid), dim3(kPassThreads), smem, st, ca->rowptr, ca->col, ca->val, ca->m,
                                    ca->n, W.z32, W.part, W.ticket, W.lvl2, pcg_vecs(W)));
    }
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

constexpr int kSmallThreads = 128;

// s = P v, one warp per row (4 rows per CTA); the last CTA to finish runs the
// epilogue.  START (v = g): r = g, dx = 0, z = s, rr = g.s and the cycle's stop
// level (the residual must drop by max(tol / (2 eta), kInnerFloor)).  STEP
// (v = r): beta step as above, one more pass counted, done once rr' <= stop.
// Factored form (rs_self): P is R^-1 and v = t = R^-T r, so s = R^-1 R^-T r
// without forming R^-1 R^-T (whose condition number kappa(R)^2 ruins it in
// FP64 beyond kappa ~ 1e7), and r.s = t.t >= 0; START then takes the residual
// from rsrc (g) rather than from v.
template <bool START>
__global__ void __launch_bounds__(kSmallThreads)
pcg_matvec(const double* __restrict__ P, int64_t n, const double* __restrict__ v, PcgVecs V,
           uint32_t* __restrict__ ticket, double tol, const double* __restrict__ rsrc, int rs_self) {
  __shared__ double red[kSmallThreads / 32];
  __shared__ double s_beta;
  __shared__ int s_last;
  grid_dep_trigger();                                // few CTAs: let the next pass launch now
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // P is read-only here: load this warp's first chunk of its first row before
  // waiting for the kernel that produced v
  double p0[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) p0[u] = (gw < n && lane + 32 * u < n) ? __ldg(P + gw * n + lane + 32 * u) : 0.0;
  grid_dep_wait();
  if (!START && V.scal[kDone] != 0.0) return;
  for (int64_t i = gw; i < n; i += nw) {
    const double* pr = P + i * n;
    double acc = 0.0;
    int64_t k = lane;
    for (; k + 224 < n; k += 256) {
      double pv[8], vv[8];
      const bool pre = (i == gw && k == lane);       // chunk already in p0
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        pv[u] = pre ? p0[u] : __ldg(pr + k + 32 * u);
        vv[u] = __ldcg(v + k + 32 * u);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = fma(pv[u], vv[u], acc);
    }
    for (; k < n; k += 32) acc = fma(__ldg(pr + k), __ldcg(v + k), acc);
    acc = warp_sum(acc);
    if (lane == 0) V.s[i] = acc;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) *ticket = 0;
  double rs = 0.0;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    const double vc = __ldcg(v + c);
    rs = fma(vc, rs_self ? vc : __ldcg(V.s + c), rs);
  }
  rs = cta_sum0(rs, red);
  if (threadIdx.x == 0) {
    if (START) {
      V.scal[kRR] = rs;
      const double eta = V.scal[kEta];
      const double want = (eta > 0.0) ? 0.5 * tol / eta : kInnerFloor;
      const double ratio = want > kInnerFloor ? want : kInnerFloor;
      V.scal[kStop2] = ratio * ratio * rs;
      V.scal[kDone] = (rs > 0.0) ? 0.0 : 1.0;
      s_beta = 0.0;
    } else {
      const double rr = V.scal[kRR];
      s_beta = (rr > 0.0) ? rs / rr : 0.0;
      V.scal[kRR] = rs;
      V.scal[kPasses] += 1.0;
      if (!(rs > V.scal[kStop2])) V.scal[kDone] = 1.0;
    }
  }
  __syncthreads();
  const double beta = s_beta;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    const double sc = __ldcg(V.s + c);
    double zc;
    if (START) {
      zc = sc;
      V.rx[c] = __ldcg((rsrc ? rsrc : v) + c);
      V.dx[c] = 0.0;
    } else {
      zc = fma(beta, V.z[c], sc);
    }
    V.z[c] = zc;
    V.z32[c] = (float)zc;
  }
}

__global__ void __launch_bounds__(kSmallThreads) pcg_apply_kernel(const double* __restrict__ dx, int64_t n,
                                                                  double* __restrict__ x) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    x[c] += dx[c];
}

// P = R^-1 R^-T from the row-major upper-triangular R^-1: P[i][j] =
// sum_{k >= max(i, j)} Rinv[i][k] Rinv[j][k].  16 x 16 output tiles of the
// upper triangle (mirrored), k in tiles of 16 through shared memory.
constexpr int kPT = 16;
__global__ void __launch_bounds__(kPT * kPT) pgram_kernel(const double* __restrict__ Rinv, int64_t n,
                                                          double* __restrict__ P) {
  __shared__ double ta[kPT][kPT + 1], tb[kPT][kPT + 1];
  const int64_t T = (n + kPT - 1) / kPT;
  int64_t idx = blockIdx.x, ti = 0;
  while (idx >= T - ti) { idx -= T - ti; ++ti; }     // upper-triangle tile (ti, tj), tj >= ti
  const int64_t tj = ti + idx;
  const int ty = threadIdx.x / kPT, tx = threadIdx.x % kPT;
  const int64_t i0 = ti * kPT, j0 = tj * kPT;
  double acc = 0.0;
  for (int64_t k0 = j0; k0 < n; k0 += kPT) {         // Rinv[j][k] = 0 for k < j0 <= j
    const int64_t ra = i0 + ty, rb = j0 + ty, kk = k0 + tx;
    ta[ty][tx] = (ra < n && kk < n) ? Rinv[ra * n + kk] : 0.0;
    tb[ty][tx] = (rb < n && kk < n) ? Rinv[rb * n + kk] : 0.0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kPT; ++u) acc = fma(ta[ty][u], tb[tx][u], acc);
    __syncthreads();
  }
  const int64_t i = i0 + ty, j = j0 + tx;
  if (i < n && j < n) {
    P[i * n + j] = acc;
    P[j * n + i] = acc;
  }
}

sns_status pgram_build(const double* Rinv, int64_t n, double* P, cudaStream_t st) {
  const int64_t T = (n + kPT - 1) / kPT;
  {
    SNS_PROF(K_RINV, st);
    pgram_kernel<<<(unsigned)(T * (T + 1) / 2), kPT * kPT, 0, st>>>(Rinv, n, P);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

static int pcg_grid(int64_t n) { return (int)std::max<int64_t>(1, (n + kSmallThreads / 32 - 1) / (kSmallThreads / 32)); }

sns_status pcg_start(const IterWs& W, int64_t n, double tol, cudaStream_t st, bool factored) {
  if (factored) {
    sns_status s = saa_matvec(W.RinvT, n, W.g, W.w, false, st);        // t = R^-T g
    if (s != SNS_OK) return s;
  }
  {
    SNS_PROF(K_MATVEC, st);
    if (factored)
      pcg_matvec<true><<<pcg_grid(n), kSmallThreads, 0, st>>>(W.Rinv, n, W.w, pcg_vecs(W), W.ticket + kPcgTicket,
                                                               tol, W.g, 1);
    else
      pcg_matvec<true><<<pcg_grid(n), kSmallThreads, 0, st>>>(W.P, n, W.g, pcg_vecs(W), W.ticket + kPcgTicket, tol,
                                                               nullptr, 0);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}
sns_status pcg_start_rhs(const IterWs& W, int64_t n, double tol, const double* v, cudaStream_t st) {
  {
    SNS_PROF(K_MATVEC, st);
    pcg_matvec<true><<<pcg_grid(n), kSmallThreads, 0, st>>>(W.P, n, v, pcg_vecs(W), W.ticket + kPcgTicket, tol,
                                                             nullptr, 0);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}
sns_status pcg_step(const IterWs& W, int64_t n, cudaStream_t st, bool factored) {
  if (factored) {
    // t = R^-T r into w (the pass's w is consumed by its own epilogue)
    sns_status s = saa_matvec(W.RinvT, n, W.rx, W.w, false, st);
    if (s != SNS_OK) return s;
  }
  {
    SNS_PROF(K_MATVEC, st);
    if (factored)
      SNS_CUDA_TRY(launch_dependent(pcg_matvec<false>, dim3(pcg_grid(n)), dim3(kSmallThreads), 0, st, W.Rinv, n,
                                    W.w, pcg_vecs(W), W.ticket + kPcgTicket, 0.0, (const double*)nullptr, 1));
    else
      SNS_CUDA_TRY(launch_dependent(pcg_matvec<false>, dim3(pcg_grid(n)), dim3(kSmallThreads), 0, st, W.P, n, W.rx,
                                    pcg_vecs(W), W.ticket + kPcgTicket, 0.0, (const double*)nullptr, 0));
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

// max |R_ii| and min |R_ii| over i < n of the column-major W (leading dim ldw).
__global__ void __launch_bounds__(kSmallThreads) diag_range_kernel(const double* __restrict__ W, int64_t ldw,
                                                                   int64_t n, double* __restrict__ out) {
  __shared__ double rmax[kSmallThreads / 32], rmin[kSmallThreads / 32];
  double mx = 0.0, mn = INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double a = fabs(W[i * ldw + i]);
    mx = fmax(mx, a);
    mn = fmin(mn, a);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    rmax[threadIdx.x >> 5] = mx;
    rmin[threadIdx.x >> 5] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kSmallThreads / 32; ++w) {
      mx = fmax(mx, rmax[w]);
      mn = fmin(mn, rmin[w]);
    }
    mx = fmax(mx, rmax[0]);
    mn = fmin(mn, rmin[0]);
    out[0] = mx;
    out[1] = mn;
  }
}
sns_status diag_range(const double* W, int64_t ldw, int64_t n, double* out, cudaStream_t st) {
  {
    SNS_PROF(K_QR, st);
    diag_range_kernel<<<1, kSmallThreads, 0, st>>>(W, ldw, n, out);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}
sns_status pcg_apply(const IterWs& W, int64_t n, double* x, cudaStream_t st) {
  {
    SNS_PROF(K_CG, st);
    pcg_apply_kernel<<<(unsigned)std::max<int64_t>(1, (n + kSmallThreads - 1) / kSmallThreads), kSmallThreads, 0,
                       st>>>(W.dx, n, x);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

// eta = ||g|| / (||A||_F ||r||) after a resid_pass; copies
// [eta, ||r||, ||g||, ||A||_F] to host_out (pinned) asynchronously.
__global__ void __launch_bounds__(kSmallThreads) eta_kernel(const double* __restrict__ g, int64_t n, double* scal) {
  __shared__ double red[kSmallThreads / 32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(g[i], g[i], s);
  s = cta_sum0(s, red);
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
    scal[12] = scal[kPasses];
  }
}
sns_status iter_reset(const IterWs& W, cudaStream_t st) {
  SNS_CUDA_TRY(cudaMemsetAsync(W.scal + kStop2, 0, 3 * sizeof(double), st));
  return SNS_OK;
}

sns_status eta_eval(const IterWs& W, int64_t n, double* host_out, cudaStream_t st) {
  {
    SNS_PROF(K_ETA, st);
  eta_kernel<<<1, kSmallThreads, 0, st>>>(W.g, n, W.scal);
  }
  SNS_LAUNCH_CHECK();
  SNS_CUDA_TRY(cudaMemcpyAsync(host_out, W.scal + 8, kHostSlots * sizeof(double), cudaMemcpyDeviceToHost, st));
  return SNS_OK;
}

}  // namespace sns
