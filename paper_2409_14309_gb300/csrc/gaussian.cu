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
#include <cstdlib>
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
  return 8192 + 256;   // the BF16 table (uploaded per call) and an error word
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

// ---------------------------------------------------------------------------
// Tensor-core path (tcgen05, BF16 operands, FP32 accumulation in TMEM).
//
// CTA tile: 256 rows of G (two M = 128 MMA tiles) x up to 256 columns of A x a
// range of K (rows of A).  Per 64-row chunk of A, all 256 threads write the
// chunk's G tile (generated from the hash and the BF16 table) and the BF16
// copy of A's chunk into shared memory in the canonical K-major layout without
// swizzle (8 x 16-byte core matrices: element (r, k) at
// ((r/8)*8 + k/8)*128 + (r%8)*16 + (k%8)*2), then one thread issues
// 2 (M tiles) x 4 (K = 16 steps) MMAs of 128 x N x 16 and commits them to the
// stage's mbarrier.  Two stages alternate, so writing chunk c+1 overlaps the
// MMAs of chunk c.  The b column is accumulated on the CUDA cores from the same
// BF16 G tile.  The epilogue reads TMEM (tcgen05.ld), scales by 1/sqrt(d) and
// adds into SA / Sb with FP32 reductions (the K range is split over CTAs).
// Waits are bounded; on expiry the CTA records an error, lets its issued MMAs
// drain (bounded), frees its TMEM and returns.
constexpr int kUG = 256;          // G rows per CTA
constexpr int kUKT = 64;          // K rows per stage
constexpr int kUN = 256;          // max columns per CTA
constexpr int kUKC = kUKT / 8;    // core matrices along K
constexpr uint32_t kUStageA = kUG * kUKT * 2;   // 32 KB
constexpr uint32_t kUStageB = kUN * kUKT * 2;   // 32 KB
constexpr long long kUWait = 1LL << 24;

SNS_D uint32_t u_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
SNS_D uint32_t kmaj_off(int r, int k) { return (uint32_t)(((r >> 3) * kUKC + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2); }
SNS_D uint64_t u_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;              // LBO: next core matrix along K
  d |= (uint64_t)(((kUKC * 128u) >> 4) & 0x3FFF) << 32;     // SBO: next 8-row group
  d |= (uint64_t)1 << 46;                                   // descriptor version
  return d;                                                 // no swizzle
}
SNS_D bool u_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kUWait; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0,1,0,p;\n\t}"
        : "=r"(ok)
        : "r"(u_smem(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
SNS_D uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(256, 1)
gauss_umma(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n, int64_t d,
           uint64_t s0, const uint16_t* __restrict__ table, int64_t kchunk, float scale, float* __restrict__ SA,
           int64_t ldsa, float* __restrict__ Sb, int64_t sbs, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t usm[];
  uint8_t* stA[2] = {usm, usm + kUStageA + kUStageB};
  uint8_t* stB[2] = {usm + kUStageA, usm + 2 * kUStageA + kUStageB};
  uint16_t* T = reinterpret_cast<uint16_t*>(usm + 2 * (kUStageA + kUStageB));   // 4096 entries
  float* bst = reinterpret_cast<float*>(T + 4096);                                 // [2][kUKT]
  __shared__ __align__(8) uint64_t mma_done[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r_base = (int64_t)blockIdx.x * kUG;            // first G row of this CTA
  const int64_t col0 = (int64_t)blockIdx.z * kUN;              // first column of A
  const int ncols = (int)min((int64_t)kUN, n - col0);
  const int npad = ((ncols + 15) / 16) * 16;                   // MMA N (multiple of 16)
  const bool with_b = (blockIdx.z == 0);
  const int64_t i_begin = (int64_t)blockIdx.y * kchunk;
  const int64_t i_end = min(m, i_begin + kchunk);
  const int64_t groups = (d + 3) / 4;
  for (int j = tid; j < 4096; j += blockDim.x) T[j] = table[j];
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(u_smem(&mma_done[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(u_smem(&mma_done[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(u_smem(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_base;
  const uint32_t idesc =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  float sb_acc = 0.f;                                            // b column, row r_base + tid
  const int64_t nchunks = (i_end - i_begin + kUKT - 1) / kUKT;
  int64_t issued = 0;                                            // chunks whose MMAs were issued
  for (int64_t c = 0; c < nchunks; ++c) {
    const int s = (int)(c & 1);
    const int64_t u = c >> 1;                                    // use index of stage s
    if (u >= 1 && !u_wait(&mma_done[s], (uint32_t)((u - 1) & 1))) {
      if (lane == 0) atomicExch(&s_fail, 1);
    }
    __syncthreads();
    if (s_fail) break;
    const int64_t i0 = i_begin + c * kUKT;
    uint8_t* sA = stA[s];
    uint8_t* sB = stB[s];
    // G tile: task (k pair, group of 4 rows): 32 x 64 tasks
    for (int t = tid; t < (kUKT / 2) * (kUG / 4); t += blockDim.x) {
      const int kp = t % (kUKT / 2), rg = t / (kUKT / 2);
      const int k0 = 2 * kp;
      const int64_t ia = i0 + k0, ib = ia + 1;
      const int64_t g = r_base / 4 + rg;
      uint64_t ka = 0, kb = 0;
      const bool oka = ia < i_end && g < groups, okb = ib < i_end && g < groups;
      if (oka) ka = splitmix_at(s0, (uint64_t)ia * (uint64_t)groups + (uint64_t)g);
      if (okb) kb = splitmix_at(s0, (uint64_t)ib * (uint64_t)groups + (uint64_t)g);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = 4 * rg + q;
        const bool rowok = r_base + r < d;
        const uint16_t va = (oka && rowok) ? T[(ka >> (16 * q + 4)) & 0xFFF] : (uint16_t)0;
        const uint16_t vb = (okb && rowok) ? T[(kb >> (16 * q + 4)) & 0xFFF] : (uint16_t)0;
        *reinterpret_cast<uint32_t*>(sA + kmaj_off(r, k0)) = (uint32_t)va | ((uint32_t)vb << 16);
      }
    }
    // A chunk: task (k pair, column) -> BF16 pair, K-major
    for (int t = tid; t < (kUKT / 2) * npad; t += blockDim.x) {
      const int nn = t % npad, kp = t / npad;
      const int k0 = 2 * kp;
      const int64_t ia = i0 + k0, ib = ia + 1;
      float fa = 0.f, fb = 0.f;
      if (nn < ncols) {
        if (ia < i_end) fa = __ldg(A + ia * lda + col0 + nn);
        if (ib < i_end) fb = __ldg(A + ib * lda + col0 + nn);
      }
      *reinterpret_cast<uint32_t*>(sB + kmaj_off(nn, k0)) = pack_bf16(fa, fb);
    }
    if (with_b && tid < kUKT) {
      const int64_t i = i0 + tid;
      bst[s * kUKT + tid] = (i < i_end) ? __bfloat162float(__float2bfloat16_rn(__ldg(b + i))) : 0.f;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int ks = 0; ks < kUKT / 16; ++ks) {
          const uint64_t ad = u_desc(u_smem(sA) + (uint32_t)mt * (kUStageA / 2) + (uint32_t)ks * 256u);
          const uint64_t bd = u_desc(u_smem(sB) + (uint32_t)ks * 256u);
          const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr + (uint32_t)mt * 256u),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       u_smem(&mma_done[s]))
                   : "memory");
    }
    issued = c + 1;
    // b column on the CUDA cores: row tid of the G tile times the BF16 b chunk
    if (with_b) {
      const float* bc = bst + s * kUKT;
#pragma unroll
      for (int k8 = 0; k8 < kUKT / 8; ++k8) {
        const uint4 w = *reinterpret_cast<const uint4*>(sA + kmaj_off(tid, 8 * k8));
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          sb_acc = fmaf(__uint_as_float(ws[h] << 16), bc[8 * k8 + 2 * h], sb_acc);
          sb_acc = fmaf(__uint_as_float(ws[h] & 0xFFFF0000u), bc[8 * k8 + 2 * h + 1], sb_acc);
        }
      }
    }
  }
  // wait for the last issued chunk's MMAs (commits track all earlier MMAs)
  bool ok = true;
  if (issued > 0) {
    const int64_t cl = issued - 1;
    ok = u_wait(&mma_done[cl & 1], (uint32_t)((cl >> 1) & 1));
  }
  __syncthreads();
  if (!ok || s_fail) {
    if (tid == 0) atomicExch(err, 1);
  } else if (issued > 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int mt = warp >> 2, quarter = warp & 3;
    const int64_t row = r_base + (int64_t)mt * 128 + quarter * 32 + lane;
    for (int c0 = 0; c0 < npad; c0 += 16) {
      uint32_t v[16];
      const uint32_t a = taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(mt * 256 + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(a));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < d) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = c0 + j;
          if (col < ncols) atomicAdd(SA + row * ldsa + col0 + col, __uint_as_float(v[j]) * scale);
        }
      }
    }
    if (with_b && r_base + tid < d) atomicAdd(Sb + (r_base + tid) * sbs, sb_acc * scale);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr) : "memory");
}

size_t gauss_umma_smem() { return 2 * (size_t)(kUStageA + kUStageB) + 4096 * 2 + 2 * kUKT * 4; }

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
  static int use_simt = -1;
  if (use_simt < 0) {
    const char* e = getenv("SNSOLVE_GAUSS");
    use_simt = (e && e[0] == 's') ? 1 : 0;
  }
  if (!use_simt) {
    int* err = reinterpret_cast<int*>(static_cast<uint8_t*>(ws) + 8192);
    SNS_CUDA_TRY(cudaMemsetAsync(err, 0, 4, st));
    const int64_t mtiles = (d + kUG - 1) / kUG;
    const int64_t ntiles = (a.n + kUN - 1) / kUN;
    int64_t ksplit = std::max<int64_t>(1, (int64_t)num_sms() / std::max<int64_t>(1, mtiles * ntiles));
    int64_t kchunk = (a.m + ksplit - 1) / ksplit;
    kchunk = ((kchunk + kUKT - 1) / kUKT) * kUKT;
    ksplit = (a.m + kchunk - 1) / kchunk;
    SNS_CUDA_TRY(raise_smem_limit((const void*)gauss_umma));
    dim3 grid((unsigned)mtiles, (unsigned)ksplit, (unsigned)ntiles);
    {
      SNS_PROF(K_GAUSS, st);
      gauss_umma<<<grid, 256, gauss_umma_smem(), st>>>(
          static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b), a.m, a.n, d,
          stream_state(seed, kStreamGaussian), dtab, kchunk, (float)(1.0 / std::sqrt((double)d)), SA, ldsa, Sb, sbs,
          err);
    }
    SNS_CUDA_TRY(cudaGetLastError());
    return SNS_OK;
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
