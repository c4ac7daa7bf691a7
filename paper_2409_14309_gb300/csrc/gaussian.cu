// Gaussian sketch (Sec. 1.2.1: dense sketch with iid Gaussian entries):
//   S [A | b] = (1/sqrt(d)) G [A | b],
// G[k, i] = T[j], j = top 12 bits of 16-bit field (k mod 4) of SplitMix64
// output i * ceil(d/4) + k/4 of stream 3, T[j] = BF16(Phi^-1((j + 1/2)/4096)).
// G is never stored: tiles are generated where they are consumed.  The operand
// [A | b] is rounded to BF16 (round to nearest even) and products accumulate in
// FP32, the precision of a BF16 tensor-core contraction.
//
// This file holds the host-side table and the SIMT reference-speed path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace sns {

// Standard normal CDF through the C library's erfc; quantile by bisection to
// full double precision (no approximation formula involved).
static double norm_cdf(double x) { return 0.5 * std::erfc(-x / std::sqrt(2.0)); }
static double norm_quantile(double p) {
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (norm_cdf(mid) < p) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}
// Nearest BF16 (8 significant bits, ties to even) of a double, as raw bits.
static uint16_t bf16_bits_rne(double x) {
  if (x == 0.0) return 0;
  int e = 0;
  const double mant = std::frexp(x, &e);                     // x = mant * 2^e, 0.5 <= |mant| < 1
  const double r = std::nearbyint(std::ldexp(mant, 8));      // default mode: ties to even
  const float f = (float)std::ldexp(r, e - 8);               // exactly representable
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}
void gauss_table_host(uint16_t* out) {
  for (int j = 0; j < 4096; ++j) out[j] = bf16_bits_rne(norm_quantile((j + 0.5) / 4096.0));
}

static uint16_t g_table[4096];
static bool g_table_ready = false;
static const uint16_t* table_host() {
  if (!g_table_ready) {
    gauss_table_host(g_table);
    g_table_ready = true;
  }
  return g_table;
}

size_t gauss_ws_bytes(int64_t m, int64_t n, int64_t d) {
  (void)m; (void)n; (void)d;
  return 4096 * 2 + 256;   // the BF16 table, uploaded per call
}

constexpr int kGMt = 64, kGNt = 64, kGKc = 32;

// Tile (kGMt x kGNt) of G[A|b] over a K range; SIMT FP32 FMAs of BF16 values.
__global__ void __launch_bounds__(256)
gauss_simt(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n, int64_t d,
           uint64_t s0, const uint16_t* __restrict__ table, int64_t kchunk, float scale, float* __restrict__ SA,
           int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  __shared__ float T[4096];
  __shared__ float Gs[kGKc][kGMt + 1];
  __shared__ float As[kGKc][kGNt + 1];
  const int tid = threadIdx.x;
  for (int j = tid; j < 4096; j += blockDim.x) T[j] = __uint_as_float((uint32_t)table[j] << 16);
  const int64_t q = n + 1;
  const int64_t ntn = (q + kGNt - 1) / kGNt;
  const int64_t tm = blockIdx.x / ntn, tn = blockIdx.x % ntn;
  const int64_t k0 = tm * kGMt, j0 = tn * kGNt;
  const int64_t i_begin = (int64_t)blockIdx.y * kchunk;
  const int64_t i_end = std::min<int64_t>(m, i_begin + kchunk);
  const int64_t groups = (d + 3) / 4;
  const int tx = tid % 16, ty = tid / 16;
  float acc[4][4] = {};
  __syncthreads();
  for (int64_t i0 = i_begin; i0 < i_end; i0 += kGKc) {
    // G tile: kGKc rows of A (i) x kGMt rows of G (k); one hash per 4 k
    for (int e = tid; e < kGKc * (kGMt / 4); e += blockDim.x) {
      const int il = e / (kGMt / 4), g4 = e % (kGMt / 4);
      const int64_t i = i0 + il;
      const int64_t kg = (k0 >> 2) + g4;
      uint64_t key = 0;
      if (i < i_end && kg < groups) key = splitmix_at(s0, (uint64_t)i * (uint64_t)groups + (uint64_t)kg);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t k = kg * 4 + t;
        const uint32_t idx = (uint32_t)((key >> (16 * t + 4)) & 0xFFFu);
        Gs[il][g4 * 4 + t] = (i < i_end && k < d) ? T[idx] : 0.f;
      }
    }
    // operand tile: BF16-rounded [A | b]
    for (int e = tid; e < kGKc * kGNt; e += blockDim.x) {
      const int il = e / kGNt, jl = e % kGNt;
      const int64_t i = i0 + il, j = j0 + jl;
      float v = 0.f;
      if (i < i_end && j < q) v = (j < n) ? A[i * lda + j] : b[i];
      As[il][jl] = __bfloat162float(__float2bfloat16_rn(v));
    }
    __syncthreads();
#pragma unroll 8
    for (int il = 0; il < kGKc; ++il) {
      float gv[4], av[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) gv[a] = Gs[il][ty * 4 + a];
#pragma unroll
      for (int c = 0; c < 4; ++c) av[c] = As[il][tx * 4 + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(gv[a], av[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t k = k0 + ty * 4 + a, j = j0 + tx * 4 + c;
      if (k < d && j < q) {
        if (j < n) atomicAdd(SA + k * ldsa + j, acc[a][c] * scale);
        else atomicAdd(Sb + k * sbs, acc[a][c] * scale);
      }
    }
}

sns_status gauss_apply_dense(const DenseArgs& a, int64_t d, uint64_t seed, float* SA, int64_t ldsa, float* Sb,
                             int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!ws || ws_bytes < gauss_ws_bytes(a.m, a.n, d)) return SNS_ENOMEM;
  uint16_t* dtab = static_cast<uint16_t*>(ws);
  SNS_CUDA_TRY(cudaMemcpyAsync(dtab, table_host(), 4096 * 2, cudaMemcpyHostToDevice, st));
  if (ldsa == a.n) {
    SNS_CUDA_TRY(cudaMemsetAsync(SA, 0, (size_t)d * a.n * 4, st));
  } else {
    SNS_CUDA_TRY(cudaMemset2DAsync(SA, (size_t)ldsa * 4, 0, (size_t)a.n * 4, (size_t)d, st));
  }
  if (sbs == 1) {
    SNS_CUDA_TRY(cudaMemsetAsync(Sb, 0, (size_t)d * 4, st));
  } else {
    SNS_CUDA_TRY(cudaMemset2DAsync(Sb, (size_t)sbs * 4, 0, 4, (size_t)d, st));
  }
  const int64_t q = a.n + 1;
  const int64_t tiles = ((d + kGMt - 1) / kGMt) * ((q + kGNt - 1) / kGNt);
  int64_t ksplit = std::max<int64_t>(1, ((int64_t)num_sms() * 6 + tiles - 1) / tiles);
  int64_t kchunk = (a.m + ksplit - 1) / ksplit;
  kchunk = ((kchunk + kGKc - 1) / kGKc) * kGKc;
  ksplit = (a.m + kchunk - 1) / kchunk;
  dim3 grid((unsigned)tiles, (unsigned)ksplit);
  {
    SNS_PROF(K_GAUSS, st);
  gauss_simt<<<grid, 256, 0, st>>>(static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b), a.m, a.n, d,
                                   stream_state(seed, kStreamGaussian), dtab, kchunk,
                                   (float)(1.0 / std::sqrt((double)d)), SA, ldsa, Sb, sbs);
  }
  SNS_CUDA_TRY(cudaGetLastError());
  return SNS_OK;
}

}  // namespace sns
