// Subsampled randomized Hadamard sketch (Sec. 1.2.1; a Hadamard-based sketch
// applied with a fast transform):
//   S [A | b] = (1/sqrt(d)) P H_{m'} D [A | b],   m' = 2^ceil(log2 m),
// H unnormalised Sylvester-Hadamard (H[p, i] = (-1)^popcount(p & i)), D the
// signs of stream 1, P the d rows of [0, m') chosen by Floyd's algorithm on
// stream 2 and sorted ascending.  Rows m..m'-1 of [A | b] are zero.
//
// H_{m'} = H_{m1} (x) H_{m2} with m2 = min(m', 1024) and the row index split as
// i = i1 * m2 + i2.  FP32 with m' >= 1024 and d <= 1024 runs as one pass
// (srht_fused_f32: each block's transform stays in shared memory and the
// sampled rows accumulate in registers); otherwise pass 1 transforms every 1024-row block over i2 (a warp
// holds one column of the block: 5 butterfly stages across its 32 registers,
// 5 across lanes by shuffles) and keeps only outputs p2 that some sampled row
// needs.  Pass 2 forms each sampled row p = p1 * m2 + p2 as
// sum_{i1} (-1)^popcount(p1 & i1) Y[i1, p2, :].
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace sns {

constexpr int kM2 = 1024;
template <typename T>
constexpr int srht_ct() { return sizeof(T) == 4 ? 16 : 8; }   // columns per pass-1 tile (3 CTAs per SM)
constexpr int kSrhtMaxD = 16384;

static int64_t np2(int64_t m) {
  int64_t p = 1;
  while (p < m) p <<= 1;
  return p;
}

// The one-pass FP32 form (srht_fused_f32) takes m' >= 1024 and d <= 1024 and
// needs no Y: one d x 16 partial per CTA, at most kFusedSlots CTAs.
constexpr int64_t kFusedMaxD = 1024;
constexpr int kFusedSlots = 256;
struct SrhtLayout {
  int64_t mp, m1, m2, q, ldy;
  bool fused;
  size_t off_sample, off_need, off_nlist, off_y, off_part, off_bits, bytes;
};
static SrhtLayout srht_layout(int64_t m, int64_t n, int64_t d, bool f64) {
  SrhtLayout L{};
  L.mp = np2(m);
  L.m2 = std::min<int64_t>(L.mp, kM2);
  L.m1 = L.mp / L.m2;
  L.q = n + 1;
  L.ldy = (L.q + 3) & ~(int64_t)3;                 // 16-byte rows for vector stores
  L.fused = !f64 && L.m2 == kM2 && d <= kFusedMaxD;
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off += (b + 255) & ~(size_t)255; return o; };
  L.off_sample = take((size_t)d * 4);
  L.off_need = take((size_t)L.m2);
  L.off_nlist = take((size_t)(L.m2 + 1) * 4);
  if (L.fused) {
    L.off_part = take((size_t)kFusedSlots * d * 16 * 4);
    L.off_bits = take((size_t)L.mp / 8);
  }
  else L.off_y = take((size_t)L.mp * L.ldy * (f64 ? 8 : 4));
  L.bytes = off;
  return L;
}
size_t srht_ws_bytes(int64_t m, int64_t n, int64_t d, bool f64) { return srht_layout(m, n, d, f64).bytes; }

// Floyd's algorithm on one CTA: keys are drawn 32 at a time by warp 0; lane 0
// runs the sequential membership test on an open-addressing set in shared
// memory; the chosen values are then bitonic-sorted.  Also marks needed p2.
__global__ void __launch_bounds__(1024)
srht_sample_kernel(int64_t mp, int64_t d, uint64_t s0, int32_t* __restrict__ sample, uint8_t* __restrict__ need,
                   int32_t* __restrict__ nlist, int64_t m2) {
  extern __shared__ __align__(16) int32_t ssm[];
  int cap = 1;
  while (cap < 2 * d) cap <<= 1;
  int32_t* table = ssm;            // cap entries, -1 = empty
  int32_t* sel = ssm + cap;        // pow2 >= d entries
  int dp = 1;
  while (dp < d) dp <<= 1;
  for (int i = threadIdx.x; i < cap; i += blockDim.x) table[i] = -1;
  for (int i = threadIdx.x; i < dp; i += blockDim.x) sel[i] = 0x7FFFFFFF;
  for (int64_t i = threadIdx.x; i < m2; i += blockDim.x) need[i] = 0;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int64_t t0 = 0; t0 < d; t0 += 32) {
      const int64_t t = t0 + lane;
      uint32_t u = 0;
      if (t < d) {
        const uint64_t key = splitmix_at(s0, (uint64_t)t);
        const uint64_t J = (uint64_t)(mp - d + t);
        u = (uint32_t)(((key & 0xFFFFFFFFull) * (J + 1)) >> 32);
      }
      for (int l = 0; l < 32 && t0 + l < d; ++l) {
        const uint32_t ul = __shfl_sync(0xffffffffu, u, l);
        if (lane == 0) {
          const uint32_t J = (uint32_t)(mp - d + t0 + l);
          // membership of ul
          uint32_t h = (uint32_t)((ul * 0x9E3779B1u) & (uint32_t)(cap - 1));
          bool found = false;
          while (table[h] != -1) {
            if ((uint32_t)table[h] == ul) { found = true; break; }
            h = (h + 1) & (cap - 1);
          }
          const uint32_t v = found ? J : ul;
          // insert v (J is never present yet: all earlier values are < J)
          uint32_t h2 = (uint32_t)((v * 0x9E3779B1u) & (uint32_t)(cap - 1));
          while (table[h2] != -1) h2 = (h2 + 1) & (cap - 1);
          table[h2] = (int32_t)v;
          sel[t0 + l] = (int32_t)v;
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  // bitonic sort of sel[0..dp)
  for (int k = 2; k <= dp; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < dp; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int32_t a = sel[i], b = sel[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { sel[i] = b; sel[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int64_t i = threadIdx.x; i < d; i += blockDim.x) {
    sample[i] = sel[i];
    need[sel[i] % m2] = 1;
  }
  __syncthreads();
  // ascending list of the needed p2 (one thread per p2; m2 <= blockDim), count at nlist[m2]
  {
    __shared__ int wcnt[32];
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    const bool f = i < m2 && need[i];
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int k = 0; k < w; ++k) base += wcnt[k];
    if (f) nlist[base + __popc(bal & ((1u << lane) - 1u))] = i;
    if (i == (int)blockDim.x - 1) nlist[m2] = base + __popc(bal);
  }
}

// The same sample for m' <= 2^20 with a bitmap of [0, m') in shared memory
// (128 KB at most).  Warp 0 draws 32 keys at a time; a batch is decided in
// parallel against the bitmap unless one of its draws could have been inserted
// by an earlier draw of the same batch (equal draws, or a draw equal to an
// earlier J), in which case lane 0 walks the batch in order.  The sorted sample
// is then read off the bitmap in ascending order (block scan of popcounts).
constexpr int64_t kSampleBitmapMax = (int64_t)1 << 20;
__global__ void __launch_bounds__(1024)
srht_sample_bitmap(int64_t mp, int64_t d, uint64_t s0, int32_t* __restrict__ sample, uint8_t* __restrict__ need,
                   int32_t* __restrict__ nlist, int64_t m2) {
  extern __shared__ __align__(16) uint32_t bits[];            // mp bits
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int nwords = (int)((mp + 31) / 32);
  for (int i = tid; i < nwords; i += blockDim.x) bits[i] = 0u;
  for (int64_t i = tid; i < m2; i += blockDim.x) need[i] = 0;
  __syncthreads();
  if (w == 0) {
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t t0 = 0; t0 < d; t0 += 32) {
      const int64_t t = t0 + lane;
      const bool valid = t < d;
      const uint32_t jbase = (uint32_t)(mp - d + t0);           // J of the batch's first draw
      uint32_t u = 0xFFFFFFFFu;
      if (valid) {
        const uint64_t key = splitmix_at(s0, (uint64_t)t);
        u = (uint32_t)(((key & 0xFFFFFFFFull) * ((uint64_t)jbase + lane + 1)) >> 32);
      }
      const unsigned peers = __match_any_sync(0xffffffffu, u);
      const bool clash = valid && ((peers & lt) != 0u || (u >= jbase && u - jbase < (uint32_t)lane));
      if (__any_sync(0xffffffffu, clash)) {
        const int cnt = (int)min((int64_t)32, d - t0);
        for (int l = 0; l < cnt; ++l) {
          const uint32_t ul = __shfl_sync(0xffffffffu, u, l);
          if (lane == 0) {
            const bool found = (bits[ul >> 5] >> (ul & 31)) & 1u;
            const uint32_t v = found ? jbase + (uint32_t)l : ul;
            bits[v >> 5] |= 1u << (v & 31);
          }
          __syncwarp();
        }
      } else if (valid) {
        const bool found = (bits[u >> 5] >> (u & 31)) & 1u;
        const uint32_t v = found ? jbase + (uint32_t)lane : u;
        atomicOr(&bits[v >> 5], 1u << (v & 31));
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // ascending read-out: thread i scans words [i * per, (i + 1) * per)
  const int per = (nwords + (int)blockDim.x - 1) / (int)blockDim.x;
  const int wb = tid * per, we = min(nwords, wb + per);
  int cnt = 0;
  for (int i = wb; i < we; ++i) cnt += __popc(bits[i]);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int pos = incl - cnt;
  for (int k = 0; k < w; ++k) pos += wsum[k];
  for (int i = wb; i < we; ++i) {
    uint32_t x = bits[i];
    while (x) {
      const int bpos = __ffs(x) - 1;
      x &= x - 1;
      const int32_t v = i * 32 + bpos;
      if (pos < d) {
        sample[pos] = v;
        need[v % m2] = 1;
      }
      ++pos;
    }
  }
  __syncthreads();
  {
    __shared__ int wcnt[32];
    const bool f = tid < m2 && need[tid];
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int base = 0;
    for (int k = 0; k < w; ++k) base += wcnt[k];
    if (f) nlist[base + __popc(bal & ((1u << lane) - 1u))] = tid;
    if (tid == (int)blockDim.x - 1) nlist[m2] = base + __popc(bal);
  }
}

static sns_status srht_sample(int64_t mp, int64_t d, uint64_t seed, int32_t* sample, uint8_t* need,
                              int32_t* nlist, int64_t m2, cudaStream_t st) {
  if (mp <= kSampleBitmapMax) {
    const size_t smem = (size_t)((mp + 31) / 32) * 4;
    SNS_CUDA_TRY(raise_smem_limit((const void*)srht_sample_bitmap));
    {
      SNS_PROF(K_SRHT_SAMPLE, st);
      srht_sample_bitmap<<<1, 1024, smem, st>>>(mp, d, stream_state(seed, kStreamSrhtSample), sample, need, nlist,
                                                m2);
    }
    SNS_LAUNCH_CHECK();
    return SNS_OK;
  }
  int cap = 1;
  while (cap < 2 * d) cap <<= 1;
  int dp = 1;
  while (dp < d) dp <<= 1;
  const size_t smem = (size_t)(cap + dp) * 4;
  SNS_CUDA_TRY(raise_smem_limit((const void*)srht_sample_kernel));
  {
    SNS_PROF(K_SRHT_SAMPLE, st);
  srht_sample_kernel<<<1, 1024, smem, st>>>(mp, d, stream_state(seed, kStreamSrhtSample), sample, need, nlist, m2);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

// Pass 1: CTA per (block i1, column tile).  Tile = m2 rows x kSrhtCT columns in
// shared memory (column-major with padding).  D is applied on load.
template <typename T>
__global__ void __launch_bounds__(256)
srht_pass1(const T* __restrict__ A, int64_t lda, const T* __restrict__ b, int64_t m, int64_t n, int64_t m2,
           int64_t ntile, uint64_t s_sign, const uint8_t* __restrict__ need, T* __restrict__ Y, int64_t ldy) {
  constexpr int kSrhtCT = srht_ct<T>();
  extern __shared__ __align__(16) uint8_t srm[];
  T* tile = reinterpret_cast<T*>(srm);          // [kSrhtCT][m2 + 1]
  T* sgn = tile + (size_t)kSrhtCT * (m2 + 1);   // [m2]
  const int64_t ldt = m2 + 1;
  const int64_t i1 = blockIdx.x / ntile;
  const int64_t c0 = (blockIdx.x % ntile) * kSrhtCT;
  const int64_t q = n + 1;
  const int ncol = (int)std::min<int64_t>(kSrhtCT, q - c0);
  const int64_t r0 = i1 * m2;
  for (int64_t rl = threadIdx.x; rl < m2; rl += blockDim.x) {
    const int64_t row = r0 + rl;
    sgn[rl] = (row < m) ? ((splitmix_at(s_sign, (uint64_t)row) >> 63) ? T(-1) : T(1)) : T(0);
  }
  __syncthreads();
  // load D [A | b] (rows coalesced along columns), 16 independent loads in
  // flight per thread before they are stored
  constexpr int kL = 16;
  for (int64_t e0 = threadIdx.x; e0 < m2 * kSrhtCT; e0 += (int64_t)blockDim.x * kL) {
    T v[kL];
#pragma unroll
    for (int u = 0; u < kL; ++u) {
      const int64_t e = e0 + (int64_t)u * blockDim.x;
      const int64_t rl = e / kSrhtCT;
      const int c = (int)(e % kSrhtCT);
      const int64_t row = r0 + rl;
      const int64_t col = c0 + c;
      v[u] = T(0);
      if (e < m2 * kSrhtCT && row < m && c < ncol) v[u] = (col < n) ? __ldg(A + row * lda + col) : __ldg(b + row);
    }
#pragma unroll
    for (int u = 0; u < kL; ++u) {
      const int64_t e = e0 + (int64_t)u * blockDim.x;
      if (e < m2 * kSrhtCT) {
        const int64_t rl = e / kSrhtCT;
        const int c = (int)(e % kSrhtCT);
        tile[(int64_t)c * ldt + rl] = sgn[rl] * v[u];
      }
    }
  }
  __syncthreads();
  // transform: one warp per column; lane holds x[k] = tile[32 k + lane]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (m2 == kM2) {
    for (int c = w; c < ncol; c += blockDim.x / 32) {
      T* col = tile + (int64_t)c * ldt;
      T x[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) x[k] = col[32 * k + lane];
#pragma unroll
      for (int s = 1; s < 32; s <<= 1)          // strides 32*s across registers
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if ((k & s) == 0) {
            const T a = x[k], bb = x[k + s];
            x[k] = a + bb;
            x[k + s] = a - bb;
          }
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {        // strides 1..16 across lanes: o - x or x + o
        const T sg = (lane & s) ? T(-1) : T(1);
#pragma unroll
        for (int k = 0; k < 32; ++k) x[k] = fma(sg, x[k], __shfl_xor_sync(0xffffffffu, x[k], s));
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) col[32 * k + lane] = x[k];
    }
  } else {
    // small m' (< 1024): plain shared-memory butterflies
    for (int64_t h = 1; h < m2; h <<= 1) {
      for (int64_t e = threadIdx.x; e < (m2 / 2) * ncol; e += blockDim.x) {
        const int c = (int)(e / (m2 / 2));
        const int64_t t = e % (m2 / 2);
        const int64_t i = (t / h) * 2 * h + (t % h);
        T* col = tile + (int64_t)c * ldt;
        const T a = col[i], bb = col[i + h];
        col[i] = a + bb;
        col[i + h] = a - bb;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // store needed outputs p2 (row-major Y[i1*m2 + p2, c0 + c])
  for (int64_t e = threadIdx.x; e < m2 * kSrhtCT; e += blockDim.x) {
    const int64_t p2 = e / kSrhtCT;
    const int c = (int)(e % kSrhtCT);
    if (c < ncol && need[p2]) Y[(r0 + p2) * ldy + c0 + c] = tile[(int64_t)c * ldt + p2];
  }
}

// In-place unnormalised 1024-point Walsh-Hadamard transform of one column by
// one warp: lane l holds x[k] = col[32 k + l]; 5 butterfly stages across the
// registers (strides 32 s), 5 across lanes by shuffles (strides 1..16).  In a
// lane stage the lane with the stride bit set keeps o - x, the other x + o:
// one FMA with a per-lane sign of +-1 (exact multiply, the sum rounded once).
SNS_D void fwht1024_warp(float* col, int lane) {
  float x[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) x[k] = col[32 * k + lane];
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1)
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if ((k & sft) == 0) {
        const float a = x[k], bb = x[k + sft];
        x[k] = a + bb;
        x[k + sft] = a - bb;
      }
#pragma unroll
  for (int sft = 1; sft < 32; sft <<= 1) {
    const float sg = (lane & sft) ? -1.f : 1.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = fmaf(sg, x[k], __shfl_xor_sync(0xffffffffu, x[k], sft));
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) col[32 * k + lane] = x[k];
}

// Pass 1 for FP32 with 1024-row blocks: 16 columns per tile; each thread loads
// 16 float4 (4 columns of 16 rows 64 apart, row pointers stepped, no per-element
// index arithmetic); tile stride 1026 so the four column groups of a warp's
// stores fall on distinct banks; only the needed rows (compact list from the
// sampler) are written back, as float4 when the tile lies inside A.
constexpr int kT1 = 16;
constexpr int kLdt1 = 1026;
__global__ void __launch_bounds__(256, 3)
srht_pass1_f32(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n,
               int64_t ntile, uint64_t s_sign, const int32_t* __restrict__ nlist, float* __restrict__ Y, int64_t ldy) {
  extern __shared__ __align__(16) float tile[];   // [kT1][kLdt1]
  __shared__ float sgn[kM2];
  const int tid = threadIdx.x;
  const int64_t i1 = blockIdx.x / ntile;
  const int64_t c0 = (blockIdx.x % ntile) * kT1;
  const int64_t q = n + 1;
  const int ncol = (int)std::min<int64_t>(kT1, q - c0);
  const int64_t r0 = i1 * kM2;
  for (int rl = tid; rl < kM2; rl += blockDim.x) {
    const int64_t row = r0 + rl;
    sgn[rl] = (row < m) ? ((splitmix_at(s_sign, (uint64_t)row) >> 63) ? -1.f : 1.f) : 0.f;
  }
  __syncthreads();
  const bool vec = c0 + kT1 <= n;                 // the whole tile lies inside A (aligned rows)
  const int rsub = tid >> 2, c4 = tid & 3;
  if (vec) {
    const float* p = A + (r0 + rsub) * lda + c0 + 4 * c4;
    const int64_t step = 64 * lda;
    float4 v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u)
      v[u] = (r0 + rsub + 64 * u < m) ? __ldg(reinterpret_cast<const float4*>(p + u * step))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int rl = rsub + 64 * u;
      const float sg = sgn[rl];
      float* t = tile + (4 * c4) * kLdt1 + rl;
      t[0] = sg * v[u].x;
      t[kLdt1] = sg * v[u].y;
      t[2 * kLdt1] = sg * v[u].z;
      t[3 * kLdt1] = sg * v[u].w;
    }
  } else {
    for (int e = tid; e < kM2 * kT1; e += blockDim.x) {
      const int rl = e / kT1, c = e % kT1;
      const int64_t row = r0 + rl, colj = c0 + c;
      float v = 0.f;
      if (c < ncol && row < m) v = (colj < n) ? __ldg(A + row * lda + colj) : __ldg(b + row);
      tile[c * kLdt1 + rl] = sgn[rl] * v;
    }
  }
  __syncthreads();
  const int lane = tid & 31, w = tid >> 5;
  for (int c = w; c < ncol; c += blockDim.x / 32) fwht1024_warp(tile + c * kLdt1, lane);
  __syncthreads();
  const int nneed = nlist[kM2];
  if (vec) {
    for (int k = rsub; k < nneed; k += 64) {
      const int p2 = nlist[k];
      const float* t = tile + (4 * c4) * kLdt1 + p2;
      *reinterpret_cast<float4*>(Y + (r0 + p2) * ldy + c0 + 4 * c4) = make_float4(t[0], t[kLdt1], t[2 * kLdt1], t[3 * kLdt1]);
    }
  } else {
    for (int e = tid; e < nneed * kT1; e += blockDim.x) {
      const int k = e / kT1, c = e % kT1;
      if (c < ncol) {
        const int p2 = nlist[k];
        Y[(r0 + p2) * ldy + c0 + c] = tile[c * kLdt1 + p2];
      }
    }
  }
}

// One pass for FP32 with 1024-row blocks and d <= 32 * SPT: CTA per (column
// tile of 16, range of blocks i1).  Per block: D [A | b] into shared memory
// (the signs from the bit array srht_sign_bits wrote)
// (rows as float4 when the tile lies in an aligned A), the 1024-point
// transform of each column (warp per column), then every sampled row k adds
// its term (-1)^popcount(p1_k & i1) Y[i1, p2_k, c] into the CTA's d x 16
// partial in shared memory (thread: column c = tid mod 16, samples tid / 16 +
// 32 j; each entry has one owner, so plain adds in block order).  The
// next block's loads are issued before the transform, so they overlap it.
// Y never leaves the SM; the CTA writes its d x 16 partial, and
// srht_fused_reduce adds the CTAs of a column tile in CTA order.
constexpr int kFT = 16;
constexpr int kFThreads = 512;

// The signs of D as bits: bit t of word w is set when row 32 w + t gets -1
// (bit 63 of its stream-1 key).  Rows past m carry no data (their loads are
// zero), so their bits do not matter.
__global__ void __launch_bounds__(256)
srht_sign_bits(int64_t nwords, uint64_t s_sign, uint32_t* __restrict__ bits) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t v = 0;
#pragma unroll 4
    for (int t = 0; t < 32; ++t) v |= (uint32_t)(splitmix_at(s_sign, (uint64_t)(32 * w + t)) >> 63) << t;
    bits[w] = v;
  }
}
struct SrhtFusedGrid {
  int nfull, gf, gb, ctas;
};
template <int SPT>
__global__ void __launch_bounds__(kFThreads, 1)
srht_fused_f32(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n,
               int64_t m1, SrhtFusedGrid fg, const uint32_t* __restrict__ sbits, const int32_t* __restrict__ sample,
               int64_t d, float* __restrict__ part) {
  extern __shared__ __align__(16) float fsm[];
  float* tile = fsm;                                             // [kFT][kLdt1]
  uint32_t* sgn = reinterpret_cast<uint32_t*>(tile + kFT * kLdt1);   // [kM2 / 32] sign bits of the block
  uint32_t* smp = sgn + kM2 / 32;                                // [d]: p1 * 1024 + p2 (p < 2^31)
  float* sacc = reinterpret_cast<float*>(smp + d);               // [d][kFT] the CTA's partial
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int bid = blockIdx.x;
  const bool full = bid < fg.nfull * fg.gf;
  const int tix = full ? bid / fg.gf : fg.nfull;
  const int g = full ? bid % fg.gf : bid - fg.nfull * fg.gf;
  const int G = full ? fg.gf : fg.gb;
  const int64_t q = n + 1;
  const int64_t c0 = (int64_t)tix * kFT;
  const int ncol = (int)min((int64_t)kFT, q - c0);
  const int64_t ib = m1 * g / G, ie = m1 * (g + 1) / G;        // this CTA's blocks
  for (int64_t k = tid; k < d; k += blockDim.x) smp[k] = (uint32_t)sample[k];
  for (int64_t e = tid; e < d * kFT; e += blockDim.x) sacc[e] = 0.f;
  const bool vec = c0 + kFT <= n && (lda & 3) == 0 && ((uintptr_t)A & 15) == 0;
  const int rsub = tid >> 2, c4 = tid & 3;                      // rows rsub + 128 u, columns 4 c4 ..
  float4 v[8];
  auto load = [&](int64_t i1) {
    const int64_t r0 = i1 * kM2;
    if (vec) {
      const float* p = A + (r0 + rsub) * lda + c0 + 4 * c4;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (r0 + rsub + 128 * u < m) ? __ldg(reinterpret_cast<const float4*>(p + (int64_t)u * 128 * lda))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t row = r0 + rsub + 128 * u;
        float e[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t col = c0 + 4 * c4 + t;
          e[t] = (row < m && col < q) ? (col < n ? __ldg(A + row * lda + col) : __ldg(b + row)) : 0.f;
        }
        v[u] = make_float4(e[0], e[1], e[2], e[3]);
      }
    }
  };
  const int cc = tid & (kFT - 1), kk = tid >> 4;
  if (ib < ie) load(ib);
  for (int64_t i1 = ib; i1 < ie; ++i1) {
    if (tid < kM2 / 32) sgn[tid] = __ldg(sbits + i1 * (kM2 / 32) + tid);
    __syncthreads();                                             // also: the previous block's tile reads are done
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int rl = rsub + 128 * u;
      const uint32_t neg = ((sgn[rl >> 5] >> (rl & 31)) & 1u) << 31;     // D: flip the sign bit
      float* t = tile + (4 * c4) * kLdt1 + rl;
      t[0] = __uint_as_float(__float_as_uint(v[u].x) ^ neg);
      t[kLdt1] = __uint_as_float(__float_as_uint(v[u].y) ^ neg);
      t[2 * kLdt1] = __uint_as_float(__float_as_uint(v[u].z) ^ neg);
      t[3 * kLdt1] = __uint_as_float(__float_as_uint(v[u].w) ^ neg);
    }
    __syncthreads();
    if (i1 + 1 < ie) load(i1 + 1);
    if (w < ncol) fwht1024_warp(tile + w * kLdt1, lane);
    __syncthreads();
    if (cc < ncol) {
      const float* col = tile + cc * kLdt1;
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        const int64_t k = kk + 32 * j;
        if (k < d) {
          const uint32_t p = smp[k];
          // (-1)^popcount(p1 & i1) applied to the sign bit (p1 = p / 1024, i1 < 2^21)
          const uint32_t neg = (uint32_t)__popc((p >> 10) & (uint32_t)i1) << 31;
          sacc[k * kFT + cc] += __uint_as_float(__float_as_uint(col[p & (kM2 - 1)]) ^ neg);
        }
      }
    }
  }
  __syncthreads();
  float* out = part + (size_t)bid * d * kFT;
  for (int64_t e = tid; e < d * kFT; e += blockDim.x) out[e] = sacc[e];
}

// SA and Sb from the fused partials: entry (k, j) of column tile j / 16 is the
// sum over that tile's CTAs, in CTA order, times 1/sqrt(d).
__global__ void __launch_bounds__(256)
srht_fused_reduce(const float* __restrict__ part, int64_t d, int64_t n, SrhtFusedGrid fg, float scale,
                  float* __restrict__ SA, int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  const int64_t q = n + 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < d * q; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / q, j = e - k * q;
    const int64_t tix = j / kFT;
    const bool full = tix < fg.nfull;
    const int64_t cta0 = full ? tix * fg.gf : (int64_t)fg.nfull * fg.gf;
    const int G = full ? fg.gf : fg.gb;
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += __ldg(part + ((size_t)(cta0 + g) * d + k) * kFT + (j - tix * kFT));
    if (j < n) SA[k * ldsa + j] = s * scale;
    else Sb[k * sbs] = s * scale;
  }
}

// Pass 2: CTA per sampled row p = p1 * m2 + p2.  Warp w adds the terms
// i1 = w, w + 8, ... of sum_{i1} (-1)^popcount(p1 & i1) Y[i1, p2, :] for 32 * kCPL
// columns at a time (kCPL per lane, kB terms' loads in flight), each as a
// compensated (TwoSum) pair; the 8 warps' pairs are then added in warp order.
constexpr int kCPL = 9;
constexpr int kP2B = 4;
template <typename T>
__global__ void __launch_bounds__(256)
srht_pass2_split(const T* __restrict__ Y, int64_t ldy, int64_t q, int64_t m1, int64_t m2,
                 const int32_t* __restrict__ sample, T scale, T* __restrict__ SA, int64_t ldsa, T* __restrict__ Sb,
                 int64_t sbs) {
  constexpr int kW = 8;
  __shared__ T shi[kW][32 * kCPL], slo[kW][32 * kCPL];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t k = blockIdx.x;
  const int64_t p = sample[k];
  const int64_t p1 = p / m2, p2 = p % m2;
  for (int64_t cb = 0; cb < q; cb += 32 * kCPL) {
    T hi[kCPL], lo[kCPL];
#pragma unroll
    for (int s = 0; s < kCPL; ++s) hi[s] = lo[s] = T(0);
    for (int64_t i0 = w; i0 < m1; i0 += (int64_t)kW * kP2B) {
      T v[kP2B][kCPL];
      bool neg[kP2B];
#pragma unroll
      for (int bb = 0; bb < kP2B; ++bb) {
        const int64_t i = i0 + (int64_t)bb * kW;
        const bool ok = i < m1;
        neg[bb] = ok && (__popcll((unsigned long long)(p1 & i)) & 1);
        const T* row = Y + ((ok ? i : 0) * m2 + p2) * ldy + cb + lane;
#pragma unroll
        for (int s = 0; s < kCPL; ++s)
          v[bb][s] = (ok && cb + lane + 32 * s < q) ? __ldg(row + 32 * s) : T(0);
      }
#pragma unroll
      for (int bb = 0; bb < kP2B; ++bb)
#pragma unroll
        for (int s = 0; s < kCPL; ++s) {
          const T x = neg[bb] ? -v[bb][s] : v[bb][s];
          const T t = hi[s] + x;
          const T bv = t - hi[s];
          lo[s] += (hi[s] - (t - bv)) + (x - bv);
          hi[s] = t;
        }
    }
#pragma unroll
    for (int s = 0; s < kCPL; ++s) {
      shi[w][lane + 32 * s] = hi[s];
      slo[w][lane + 32 * s] = lo[s];
    }
    __syncthreads();
    for (int cc = threadIdx.x; cc < 32 * kCPL && cb + cc < q; cc += blockDim.x) {
      T h = shi[0][cc], l = slo[0][cc];
      for (int ww = 1; ww < kW; ++ww) {
        const T x = shi[ww][cc];
        const T t = h + x;
        const T bv = t - h;
        l += ((h - (t - bv)) + (x - bv)) + slo[ww][cc];
        h = t;
      }
      const T r = (h + l) * scale;
      const int64_t c = cb + cc;
      if (c < q - 1) SA[k * ldsa + c] = r;
      else Sb[k * sbs] = r;
    }
    __syncthreads();
  }
}

// Column tiles of 16 and their CTA groups for srht_fused_f32: the full tiles
// get gf CTAs each and a last partial tile (holding b) the SMs left.  A block
// of the partial tile costs about half a full one (measured: 2.9 vs 6.3 us),
// so it counts as half a tile when the SMs are shared out.
static SrhtFusedGrid srht_fused_grid(int64_t q, int64_t m1) {
  SrhtFusedGrid fg{};
  const int sms = std::min(num_sms(), kFusedSlots);
  const int nfull = (int)(q / kFT);
  const bool rem = q % kFT != 0;
  fg.nfull = nfull;
  if (nfull == 0) {
    fg.gf = 1;
    fg.gb = sms;
  } else if (!rem) {
    fg.gf = std::max(1, sms / nfull);
  } else {
    fg.gf = std::max(1, (2 * sms) / (2 * nfull + 1));
    fg.gb = std::max(1, sms - nfull * fg.gf);
  }
  fg.gf = (int)std::min<int64_t>(fg.gf, m1);
  fg.gb = (int)std::min<int64_t>(fg.gb, m1);
  fg.ctas = nfull * fg.gf + (rem ? fg.gb : 0);
  return fg;
}

template <int SPT>
static sns_status srht_fused_launch(const DenseArgs& a, const SrhtLayout& L, const SrhtFusedGrid& fg,
                                    const uint32_t* sbits, const int32_t* sample, int64_t d, float* part,
                                    cudaStream_t st) {
  const size_t smem = ((size_t)kFT * kLdt1 + kM2 / 32) * 4 + (size_t)d * 4 + (size_t)d * kFT * 4;
  SNS_CUDA_TRY(raise_smem_limit((const void*)srht_fused_f32<SPT>));
  {
    SNS_PROF(K_SRHT_PASS1, st);
    srht_fused_f32<SPT><<<(unsigned)fg.ctas, kFThreads, smem, st>>>(static_cast<const float*>(a.A), a.lda,
                                                                     static_cast<const float*>(a.b), a.m, a.n, L.m1,
                                                                     fg, sbits, sample, d, part);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

template <typename T>
static sns_status srht_run(const DenseArgs& a, int64_t d, uint64_t seed, T* SA, int64_t ldsa, T* Sb, int64_t sbs,
                           uint8_t* ws, const SrhtLayout& L, cudaStream_t st) {
  int32_t* sample = reinterpret_cast<int32_t*>(ws + L.off_sample);
  uint8_t* need = ws + L.off_need;
  int32_t* nlist = reinterpret_cast<int32_t*>(ws + L.off_nlist);
  T* Y = reinterpret_cast<T*>(ws + L.off_y);
  sns_status s = srht_sample(L.mp, d, seed, sample, need, nlist, L.m2, st);
  if (s != SNS_OK) return s;
  const uint64_t s_sign = stream_state(seed, kStreamSrhtSign);
  if constexpr (sizeof(T) == 4) {
    if (L.fused) {
      const SrhtFusedGrid fg = srht_fused_grid(L.q, L.m1);
      if (fg.ctas > kFusedSlots) return SNS_EINVAL;
      float* part = reinterpret_cast<float*>(ws + L.off_part);
      uint32_t* sbits = reinterpret_cast<uint32_t*>(ws + L.off_bits);
      {
        SNS_PROF(K_SRHT_SAMPLE, st);
        srht_sign_bits<<<(unsigned)std::min<int64_t>((L.mp / 32 + 255) / 256, num_sms() * 8), 256, 0, st>>>(
            L.mp / 32, s_sign, sbits);
      }
      SNS_LAUNCH_CHECK();
      s = d <= 256   ? srht_fused_launch<8>(a, L, fg, sbits, sample, d, part, st)
          : d <= 512 ? srht_fused_launch<16>(a, L, fg, sbits, sample, d, part, st)
                     : srht_fused_launch<32>(a, L, fg, sbits, sample, d, part, st);
      if (s != SNS_OK) return s;
      {
        SNS_PROF(K_SRHT_PASS2, st);
        srht_fused_reduce<<<num_sms() * 4, 256, 0, st>>>(part, d, a.n, fg, (float)(1.0 / std::sqrt((double)d)), SA,
                                                         ldsa, Sb, sbs);
      }
      SNS_LAUNCH_CHECK();
      return SNS_OK;
    }
  }
  const bool fast = sizeof(T) == 4 && L.m2 == kM2 && a.lda % 4 == 0 && (uintptr_t)a.A % 16 == 0;
  if (fast) {
    const int64_t ntile = (L.q + kT1 - 1) / kT1;
    const size_t smem = (size_t)kT1 * kLdt1 * 4;
    SNS_CUDA_TRY(raise_smem_limit((const void*)srht_pass1_f32));
    {
      SNS_PROF(K_SRHT_PASS1, st);
      srht_pass1_f32<<<(unsigned)(L.m1 * ntile), 256, smem, st>>>(
          static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b), a.m, a.n, ntile, s_sign, nlist,
          reinterpret_cast<float*>(Y), L.ldy);
    }
  } else {
    constexpr int kSrhtCT = srht_ct<T>();
    const int64_t ntile = (L.q + kSrhtCT - 1) / kSrhtCT;
    const size_t smem = ((size_t)kSrhtCT * (L.m2 + 1) + L.m2) * sizeof(T);
    SNS_CUDA_TRY(raise_smem_limit((const void*)srht_pass1<T>));
    {
      SNS_PROF(K_SRHT_PASS1, st);
      srht_pass1<T><<<(unsigned)(L.m1 * ntile), 256, smem, st>>>(static_cast<const T*>(a.A), a.lda,
                                                                static_cast<const T*>(a.b), a.m, a.n, L.m2, ntile,
                                                                s_sign, need, Y, L.ldy);
    }
  }
  SNS_LAUNCH_CHECK();
  {
    SNS_PROF(K_SRHT_PASS2, st);
    srht_pass2_split<T><<<(unsigned)d, 256, 0, st>>>(Y, L.ldy, L.q, L.m1, L.m2, sample,
                                                    (T)(1.0 / std::sqrt((double)d)), SA, ldsa, Sb, sbs);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

sns_status srht_apply_dense(const DenseArgs& a, int64_t d, uint64_t seed, void* SA, int64_t ldsa, void* Sb,
                            int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st) {
  const SrhtLayout L = srht_layout(a.m, a.n, d, a.f64);
  if (ws_bytes < L.bytes || !ws) return SNS_ENOMEM;
  if (d > kSrhtMaxD) return SNS_EINVAL;
  if (a.f64)
    return srht_run<double>(a, d, seed, static_cast<double*>(SA), ldsa, static_cast<double*>(Sb), sbs,
                            static_cast<uint8_t*>(ws), L, st);
  return srht_run<float>(a, d, seed, static_cast<float*>(SA), ldsa, static_cast<float*>(Sb), sbs,
                         static_cast<uint8_t*>(ws), L, st);
}

__global__ void widen_i32(const int32_t* in, int64_t n, int64_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

sns_status debug_srht_sample(int64_t mp, int64_t d, uint64_t seed, int64_t* out, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
  const int64_t m2 = std::min<int64_t>(mp, kM2);
  const size_t o_need = ((size_t)d * 4 + 255) / 256 * 256;
  const size_t o_list = o_need + ((size_t)m2 + 255) / 256 * 256;
  const size_t need = o_list + (size_t)(m2 + 1) * 4;
  if (!ws || ws_bytes < need || d > kSrhtMaxD) return SNS_ENOMEM;
  int32_t* sample = static_cast<int32_t*>(ws);
  uint8_t* nd = static_cast<uint8_t*>(ws) + o_need;
  int32_t* nl = reinterpret_cast<int32_t*>(static_cast<uint8_t*>(ws) + o_list);
  sns_status s = srht_sample(mp, d, seed, sample, nd, nl, m2, st);
  if (s != SNS_OK) return s;
  {
    SNS_PROF(K_MISC, st);
  widen_i32<<<64, 256, 0, st>>>(sample, d, out);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

}  // namespace sns
