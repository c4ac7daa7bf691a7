// Gaussian sketch (Sec. 1.2.1: dense sketch with iid Gaussian entries):
//   S [A | b] = (1/sqrt(d)) G [A | b],
// G[k, i] = T[j], j = byte (i mod 8) of SplitMix64 output (i div 8) * d + k of
// stream 3 (one output serves the eight columns 8t .. 8t + 7 of row k), and
// T[j] = BF16(Phi^-1((j + 1/2)/256)).
// G is never stored: tiles are generated where they are consumed.  The operand
// [A | b] enters the BF16 tensor cores as T BF16 terms (T = 1: rounded to BF16,
// round to nearest even; T = 3: the FP32 values exactly) and products
// accumulate in FP32.
//
// This file holds the host-side table, the SIMT path (one term) and the
// tensor-core path.
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
  for (int j = 0; j < kGaussLevels; ++j) out[j] = bf16_bits_rne(norm_quantile((j + 0.5) / kGaussLevels));
}

static uint16_t g_table[kGaussLevels];
static bool g_table_ready = false;
static const uint16_t* table_host() {
  if (!g_table_ready) {
    gauss_table_host(g_table);
    g_table_ready = true;
  }
  return g_table;
}

size_t gauss_err_offset() { return 8192; }

constexpr int kGMt = 64, kGNt = 64, kGKc = 32;

// Tile (kGMt x kGNt) of G[A|b] over a K range; SIMT FP32 FMAs of BF16 values.
__global__ void __launch_bounds__(256)
gauss_simt(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n, int64_t d,
           uint64_t s0, const uint16_t* __restrict__ table, int64_t kchunk, float scale, float* __restrict__ SA,
           int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  __shared__ float T[kGaussLevels];
  __shared__ float Gs[kGKc][kGMt + 1];
  __shared__ float As[kGKc][kGNt + 1];
  const int tid = threadIdx.x;
  for (int j = tid; j < kGaussLevels; j += blockDim.x) T[j] = __uint_as_float((uint32_t)table[j] << 16);
  const int64_t q = n + 1;
  const int64_t ntn = (q + kGNt - 1) / kGNt;
  const int64_t tm = blockIdx.x / ntn, tn = blockIdx.x % ntn;
  const int64_t k0 = tm * kGMt, j0 = tn * kGNt;
  const int64_t i_begin = (int64_t)blockIdx.y * kchunk;
  const int64_t i_end = std::min<int64_t>(m, i_begin + kchunk);
  const int tx = tid % 16, ty = tid / 16;
  float acc[4][4] = {};
  __syncthreads();
  for (int64_t i0 = i_begin; i0 < i_end; i0 += kGKc) {
    // G tile: kGKc rows of A (i) x kGMt rows of G (k); one hash per row k and
    // 8 consecutive i (i0 is a multiple of 8)
    for (int e = tid; e < (kGKc / 8) * kGMt; e += blockDim.x) {
      const int g8 = e / kGMt, kl = e % kGMt;
      const int64_t i = i0 + 8 * g8, k = k0 + kl;
      const uint64_t key = (i < i_end && k < d) ? splitmix_at(s0, (uint64_t)(i >> 3) * (uint64_t)d + (uint64_t)k) : 0;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        Gs[8 * g8 + t][kl] = (i + t < i_end && k < d) ? T[(uint32_t)(key >> (8 * t)) & 0xFFu] : 0.f;
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
// Two kernels.  gauss_convert streams [A | b] once and writes ready-made MMA
// operand tiles, one per (chunk of KT rows, 256-column tile), in the canonical
// K-major layout without swizzle (8 x 16-byte core matrices: element (column
// nn, row k) at ((nn/8)*(KT/8) + k/8)*128 + (nn%8)*16 + (k%8)*2), beside the
// chunk's KT b values as FP32.  A is written as T BF16 terms, T = 1, 2 or 3:
// term 1 is A rounded to BF16 (round to nearest even), term t + 1 is the
// rounding of what terms 1..t leave over; each remainder is exact in FP32
// (Sterbenz), and three terms hold an FP32 value exactly (8 + 8 + 8
// significant bits), so T = 3 multiplies the FP32 A itself.  gauss_umma then
// never touches FP32 A.  It is warp-specialised: 16 warps generate the chunk's
// 128 x KT tile of G into a 2-stage ring, and one warp takes each chunk's
// tile with bulk copies into a ring of A stages (issued stages - 1 chunks
// ahead) and issues T MMAs of 128 x N x 16 per K = 16 step, all T with the
// same G operand; the roles meet only at mbarriers.  Every A tile is read by
// the d / 128 row-tile CTAs of its K range, mostly from L2.  One term uses
// chunks of KT = 64 rows; split A uses KT = 32 so that T-fold tiles still
// leave room for a ring of A stages in shared memory.
//
// G: one hash per (row, 8 consecutive k) gives 8 lookups in a per-bank copy of
// the FP32 table and one 16-byte store; the b column is accumulated on the CUDA
// cores from the same looked-up values.
//
// Accumulation.  The tensor cores add into the TMEM accumulator in FP32
// without round-to-nearest (measured: relative error ~2^-24 per accumulated
// MMA, growing linearly with the MMAs of one accumulation run).  So the
// accumulator D (TMEM columns 0..255) only ever holds about 32 MMAs (measured
// at 2^20 x 256, d = 1024: 5.3e-7 relative error for one term, 6.6e-7 for
// three, against 3.6e-7 / 6.2e-7 with runs of 16 and 5 % / 9 % more time): then the
// CTA's warps add D into a running FP32 sum S held in TMEM columns 256..511
// (tcgen05.ld of both, round-to-nearest adds in registers, tcgen05.st of S)
// and the next chunk restarts D.  The epilogue adds D and S, scales by
// 1/sqrt(d) and stores the CTA's partial into its K split's slice of the
// workspace; gauss_reduce adds the slices in split order.
// Waits are bounded; on expiry the CTA records an error, lets its issued
// copies and MMAs land (bounded), frees its TMEM and returns.
constexpr int kUG = 128;          // G rows per CTA (one M = 128 tile)
constexpr int kUN = 256;          // max columns per CTA
constexpr uint32_t kUSum = 256;   // TMEM column of the running sum S
constexpr long long kUWait = 1LL << 24;
constexpr int kUFlushMmas = 32;   // MMAs per accumulation run in D

// Shape of the variant with T BF16 terms of A, G ring depth GS and A ring depth BS.
template <int T, int GS = 2, int BS = (T == 3 ? 3 : 5)>
struct GShape {
  static constexpr int KT = T == 1 ? 64 : 32;             // K rows per chunk
  static constexpr int KC = KT / 8;                       // core matrices along K
  static constexpr int GStages = GS;                      // G ring: chunks generated ahead of their MMAs
  static constexpr int BStages = BS;                      // A ring
  static constexpr uint32_t StageA = kUG * KT * 2;        // G tile (BF16)
  static constexpr uint32_t Term = kUN * KT * 2;          // one BF16 term of the A tile
  static constexpr uint32_t StageBb = KT * 4;             // b values of the chunk (FP32)
  static constexpr uint32_t BStage = T * Term + StageBb;  // one A stage = one converted tile (16-byte multiple)
  static constexpr int Flush = kUFlushMmas / (T * KT / 16) > 0 ? kUFlushMmas / (T * KT / 16) : 1;  // chunks per run
  static constexpr size_t Smem = (size_t)GStages * StageA + (size_t)BStages * BStage + (size_t)kGaussLevels * 32 * 4;
  static_assert(BStage % 16 == 0 && Smem <= 227 * 1024, "A stages must fit in shared memory");
};

SNS_D uint32_t u_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int KC>
SNS_D uint32_t kmaj_off(int r, int k) { return (uint32_t)(((r >> 3) * KC + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2); }
template <int KC>
SNS_D uint64_t u_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;              // LBO: next core matrix along K
  d |= (uint64_t)(((KC * 128u) >> 4) & 0x3FFF) << 32;       // SBO: next 8-row group
  d |= (uint64_t)1 << 46;                                   // descriptor version
  return d;                                                 // no swizzle
}
// Bounded wait on an mbarrier phase.  Each try suspends the thread until the
// phase completes or kUSuspendNs pass (a waiting warp then takes no issue
// slots from the working ones); kUWait tries bound the wait (~17 s).
constexpr uint32_t kUSuspendNs = 1000;
SNS_D bool u_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kUWait; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0,1,0,p;\n\t}"
        : "=r"(ok)
        : "r"(u_smem(bar)), "r"(parity), "r"(kUSuspendNs)
        : "memory");
    if (ok) return true;
  }
  return false;
}
SNS_D uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
// 16 consecutive TMEM columns of this warp's 32 lanes (32x32b shape).
SNS_D void tmem_ld16(uint32_t a, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(a));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
SNS_D void tmem_st16(uint32_t a, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(a),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
SNS_D void u_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(u_smem(bar)), "r"(bytes) : "memory");
}
SNS_D void u_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(u_smem(dst)),
      "l"(src), "r"(bytes), "r"(u_smem(bar))
      : "memory");
}

// Stage and phase parity of a ring position, advanced one chunk at a time (no
// divisions in the chunk loops).
template <int N>
struct RingPos {
  int s = 0;
  uint32_t ph = 0;
  SNS_D void next() {
    if (++s == N) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// The T BF16 terms of an FP32 value: x[0] = RN(v), x[t] = RN(v - x[0] - ..
// - x[t-1]) (every remainder exact in FP32).  Returns x[0] + .. + x[T-1] as
// FP32 (exact: v itself for T = 3 in the normal range).
template <int T>
SNS_D float bf16_terms(float v, float (&x)[T]) {
  float rem = v, sum = 0.f;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    x[t] = __bfloat162float(__float2bfloat16_rn(rem));
    rem -= x[t];
    sum += x[t];
  }
  return sum;
}

// [A | b] -> BF16 operand tiles.  Tile (chunk c, column tile z) lives at
// tiles + (c * ntiles + z) * BStage: T K-major BF16 blocks (one per term) of
// rows KT c .. KT c + KT - 1 and columns 256z .. 256z + 255 (zero past m and
// n), then (z = 0 only meaningful) the chunk's KT b values as the sum of their
// T terms, in FP32.  A block converts whole tiles; a thread takes 8 rows x 4
// columns (16-byte loads that consecutive threads make for consecutive column
// quads) and writes each term's 4 columns' 8-row runs as 16-byte stores.
template <int T>
__global__ void __launch_bounds__(256)
gauss_convert(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n,
              int64_t nchunks, int64_t ntiles, uint8_t* __restrict__ tiles) {
  using S = GShape<T>;
  const bool vec = (lda & 3) == 0 && ((uintptr_t)A & 15) == 0;
  const int64_t units = nchunks * ntiles;
  for (int64_t ct = blockIdx.x; ct < units; ct += gridDim.x) {
    const int64_t c = ct / ntiles, z = ct - c * ntiles;
    uint8_t* tile = tiles + (size_t)ct * S::BStage;
    const int64_t r0 = c * S::KT;
    for (int t = threadIdx.x; t < S::KC * (kUN / 4); t += blockDim.x) {
      const int nn = 4 * (t % (kUN / 4)), k8 = t / (kUN / 4);
      const int64_t col = z * kUN + nn;
      float f[8][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int64_t row = r0 + 8 * k8 + j;
        if (vec && row < m && col + 3 < n) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(A + row * lda + col));
          f[j][0] = v.x;
          f[j][1] = v.y;
          f[j][2] = v.z;
          f[j][3] = v.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) f[j][q] = (row < m && col + q < n) ? __ldg(A + row * lda + col + q) : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float x[8][T];
#pragma unroll
        for (int j = 0; j < 8; ++j) bf16_terms<T>(f[j][q], x[j]);
#pragma unroll
        for (int p = 0; p < T; ++p) {
          uint4 w;
          w.x = pack_bf16(x[0][p], x[1][p]);
          w.y = pack_bf16(x[2][p], x[3][p]);
          w.z = pack_bf16(x[4][p], x[5][p]);
          w.w = pack_bf16(x[6][p], x[7][p]);
          *reinterpret_cast<uint4*>(tile + (size_t)p * S::Term + kmaj_off<S::KC>(nn + q, 8 * k8)) = w;
        }
      }
    }
    if (threadIdx.x < S::KT) {
      const int64_t row = r0 + threadIdx.x;
      float x[T];
      reinterpret_cast<float*>(tile + (size_t)T * S::Term)[threadIdx.x] =
          (row < m && z == 0) ? bf16_terms<T>(__ldg(b + row), x) : 0.f;
    }
  }
}

// Warp roles: warps 0..GW-1 generate G (and the b column) and move D into S
// at the flush points; warp GW issues the MMAs and the tile copies.  They meet
// only at mbarriers: tile_ready (copy landed), g_ready (all GW generator warps
// arrived: the chunk's G tile is written and, at a flush point, D has been
// added into S), gfree / bfree (the chunk's MMAs completed: its G stage / A
// stage may be refilled; two commits after each chunk).  Phases never alias:
// a barrier's next phase cannot complete before its current one was waited for.
constexpr int kUGenWarps = 16;   // 32 would exceed 1024 threads with the MMA warp
template <int T, int GS, int BS>
__global__ void __launch_bounds__(32 * (kUGenWarps + 1), 1)
gauss_umma(const uint8_t* __restrict__ tiles, int64_t ntiles, int64_t m, int64_t n, int64_t d, uint64_t s0,
           const uint16_t* __restrict__ table, int64_t kchunk, float scale, float* __restrict__ part,
           float* __restrict__ partb, int* __restrict__ err, int flush_every) {
  using S = GShape<T, GS, BS>;
  constexpr int KT = S::KT, GST = S::GStages, BST = S::BStages;
  extern __shared__ __align__(1024) uint8_t usm[];
  // G stages (StageA each), then A stages (T terms, then the b values)
  auto stA = [&](int s) { return usm + (size_t)s * S::StageA; };
  auto stB = [&](int s) { return usm + (size_t)GST * S::StageA + (size_t)s * S::BStage; };
  auto stb = [&](int s) { return reinterpret_cast<const float*>(stB(s) + (size_t)T * S::Term); };
  // the table as FP32, replicated once per bank: entry j of lane l at sT[j * 32 + l],
  // so a warp's 32 random lookups never conflict
  float* sT = reinterpret_cast<float*>(usm + (size_t)GST * S::StageA + (size_t)BST * S::BStage);
  __shared__ __align__(8) uint64_t tile_ready[BST];     // copy of chunk c landed (stage c mod BST)
  __shared__ __align__(8) uint64_t bfree[BST];          // MMAs of chunk c done (A stage reusable)
  __shared__ __align__(8) uint64_t g_ready[GST];        // G tile of chunk c written (stage c mod GST)
  __shared__ __align__(8) uint64_t gfree[GST];          // MMAs of chunk c done (G stage reusable)
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = (warp == kUGenWarps);
  const int64_t r_base = (int64_t)blockIdx.x * kUG;            // first G row of this CTA
  const int64_t z = blockIdx.z;                                // column tile
  const int64_t col0 = z * kUN;                                // first column of A
  const int ncols = (int)min((int64_t)kUN, n - col0);
  const int npad = ((ncols + 15) / 16) * 16;                   // MMA N (multiple of 16)
  const bool with_b = (z == 0);
  const int64_t i_begin = (int64_t)blockIdx.y * kchunk;        // a multiple of KT
  const int64_t i_end = min(m, i_begin + kchunk);
  const int64_t nchunks = (i_end - i_begin + KT - 1) / KT;
  const int64_t c_base = i_begin / KT;                         // global chunk index of chunk 0
  const uint32_t term_bytes = (uint32_t)npad * KT * 2u;        // the used prefix of one term block
  const uint32_t copy_bytes = T * term_bytes + (with_b ? S::StageBb : 0u);
  for (int j = tid; j < kGaussLevels * 32; j += blockDim.x) sT[j] = __uint_as_float((uint32_t)table[j >> 5] << 16);
  if (tid == 0) {
    for (int s = 0; s < BST; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(u_smem(&tile_ready[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(u_smem(&bfree[s])) : "memory");
    }
    for (int s = 0; s < GST; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(u_smem(&g_ready[s])), "r"(kUGenWarps) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(u_smem(&gfree[s])) : "memory");
    }
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
  auto fail = [&]() { s_fail = 1; };

  // D (columns 0..255) -> S (columns kUSum..), by the generator warps: warp w
  // reads TMEM lanes of quadrant w mod 4 (the hardware rule) and the 16-column
  // blocks w / 4, w / 4 + 4, ...; the final pass adds D and S, scales and
  // stores the CTA's partial tile into its K split's slice of `part` (row
  // stride n), and each generator thread its b-column partial into `partb`
  // (slice (K split, thread group)); gauss_reduce adds the slices in a fixed
  // order.  nflush counts the flushes done (uniform over the warps).
  int nflush = 0;
  float sb_hi = 0.f, sb_lo = 0.f;                              // b column (generator threads)
  auto tmem_flush = [&](bool final_pass) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int quarter = warp & 3, cblk = warp >> 2;
    const int rloc = quarter * 32 + lane;
    const int64_t row = r_base + rloc;
    const uint32_t lanes = (uint32_t)(quarter * 32) << 16;
    for (int c0 = cblk * 16; c0 < npad; c0 += 16 * (kUGenWarps / 4)) {
      float v[16];
      tmem_ld16(taddr + lanes + (uint32_t)c0, v);
      if (nflush > 0) {
        float sacc[16];
        tmem_ld16(taddr + lanes + kUSum + (uint32_t)c0, sacc);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += sacc[j];
      }
      if (!final_pass) {
        tmem_st16(taddr + lanes + kUSum + (uint32_t)c0, v);
        continue;
      }
      if (row < d) {
        float* dst = part + ((int64_t)blockIdx.y * d + row) * n + col0 + c0;
        if (c0 + 16 <= ncols && ((uintptr_t)dst & 15) == 0) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(dst + j) =
                make_float4(v[j] * scale, v[j + 1] * scale, v[j + 2] * scale, v[j + 3] * scale);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < ncols) dst[j] = v[j] * scale;
        }
      }
    }
    if (final_pass) {
      constexpr int kGroups = 32 * kUGenWarps / kUG;             // generator threads per row of G
      if (with_b && r_base + (tid & (kUG - 1)) < d)
        partb[((int64_t)blockIdx.y * kGroups + (tid >> 7)) * d + r_base + (tid & (kUG - 1))] = (sb_hi + sb_lo) * scale;
    } else {
      ++nflush;
    }
  };

  __shared__ long long s_issued;                               // chunks whose MMAs the MMA warp issued
  if (mma_warp) {
    if (lane == 0) {
      // chunk c's tile (T terms and the b values) into A stage c mod BST
      int64_t copied = 0;
      RingPos<BST> cpos;                                         // chunk `copied` in the A ring
      auto issue_copy = [&](int64_t c) {
        const int s = cpos.s;
        cpos.next();
        const uint8_t* src = tiles + (size_t)((c_base + c) * ntiles + z) * S::BStage;
        u_expect(&tile_ready[s], copy_bytes);
#pragma unroll
        for (int p = 0; p < T; ++p) u_copy(stB(s) + (size_t)p * S::Term, src + (size_t)p * S::Term, term_bytes, &tile_ready[s]);
        if (with_b) u_copy(stB(s) + (size_t)T * S::Term, src + (size_t)T * S::Term, S::StageBb, &tile_ready[s]);
        copied = c + 1;
      };
      for (int64_t c = 0; c < BST - 1 && c < nchunks; ++c) issue_copy(c);
      int64_t issued = 0;
      int since = 0;                                             // chunks in D since the last flush
      RingPos<GST> g;                                            // chunk c in the G ring
      RingPos<BST> t, tp;                                        // chunk c and c - 1 in the A ring
      for (int64_t c = 0; c < nchunks; ++c) {
        const int sg = g.s, s = t.s;
        if (!u_wait(&g_ready[sg], g.ph)) { fail(); break; }
        if (s_fail) break;
        if (since == flush_every) since = 0;                     // D was moved into S
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int ks = 0; ks < KT / 16; ++ks) {
          const uint64_t ad = u_desc<S::KC>(u_smem(stA(sg)) + (uint32_t)ks * 256u);
#pragma unroll
          for (int p = 0; p < T; ++p) {
            const uint64_t bd = u_desc<S::KC>(u_smem(stB(s)) + (uint32_t)p * S::Term + (uint32_t)ks * 256u);
            const uint32_t acc = (since > 0 || ks > 0 || p > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         u_smem(&gfree[sg]))
                     : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         u_smem(&bfree[s]))
                     : "memory");
        issued = c + 1;
        ++since;
        // the copy BST - 1 chunks ahead goes into the A stage chunk c - 1 used
        const int64_t cn = c + BST - 1;
        if (cn < nchunks) {
          if (c >= 1 && !u_wait(&bfree[tp.s], tp.ph)) {
            fail();
            break;
          }
          issue_copy(cn);
        }
        tp = t;
        g.next();
        t.next();
      }
      s_issued = issued;
      // the last issued chunk's commit tracks all earlier MMAs; TMEM stays allocated until then
      if (issued > 0 && !u_wait(&bfree[(issued - 1) % BST], (uint32_t)(((issued - 1) / BST) & 1)))
        fail();
      // copies issued but never consumed (failure path) land before the CTA exits: a
      // stage's copies complete in order, so its last one covers the earlier ones
      for (int64_t c = max((int64_t)0, copied - BST); c < copied; ++c)
        if (!u_wait(&tile_ready[c % BST], (uint32_t)((c / BST) & 1))) fail();
    }
    __syncwarp();
  } else {
    // generator warps.  Thread (r, q) hashes outputs (i_begin / 8 + (KT / 8) c + q) d + r_base + r
    // of the stream, q = tid / 128 + e * (threads / 128): the counter state advances by
    // (KT / 8) d gamma per chunk
    constexpr int kGenThreads = 32 * kUGenWarps;
    constexpr int kPer = (KT / 8) / (kGenThreads / kUG);         // hashes per thread and chunk
    static_assert(kPer >= 1 && kPer * (kGenThreads / kUG) == KT / 8, "generator threads must tile the chunk");
    const int r = tid & (kUG - 1);
    uint64_t state[kPer];
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const uint64_t q = (uint64_t)((tid >> 7) + e * (kGenThreads / kUG));
      state[e] = s0 + (((uint64_t)(i_begin >> 3) + q) * (uint64_t)d + (uint64_t)(r_base + r) + 1) * kGamma;
    }
    const uint64_t state_step = (uint64_t)(KT / 8) * (uint64_t)d * kGamma;
    int since = 0;                                               // chunks in D since the last flush
    RingPos<GST> g, gp;                                          // chunk c and c - 1 in the G ring
    RingPos<BST> t;                                              // chunk c in the A ring
    for (int64_t c = 0; c < nchunks; ++c) {
      const int sg = g.s, s = t.s;
      // G stage sg is free once chunk c - GST's MMAs are done (the phase before
      // g.ph); the b values come with the tile
      const bool ok = (c < GST || u_wait(&gfree[sg], g.ph ^ 1u)) && u_wait(&tile_ready[s], t.ph);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) fail();
        break;
      }
      uint8_t* sA = stA(sg);
      // G tile and b column: task (row r, group q of 8 consecutive k), kPer per
      // thread: one hash gives the row's 8 entries (byte t of output
      // (i div 8) d + k is entry i = 8 (i0 / 8 + q) + t), 8 conflict-free table
      // lookups, one 16-byte store into the K-major tile, and 8 FMAs of the b
      // column in the same registers.  Rows past d and columns past m need no
      // masking: their products never reach SA (rows past d are not written out;
      // the converted A and b are zero there).
      {
        const float* bc = stb(s);
        float bpart = 0.f;
#pragma unroll
        for (int e = 0; e < kPer; ++e) {
          const int q = (tid >> 7) + e * (kGenThreads / kUG);
          const uint64_t key = mix64(state[e]);
          state[e] += state_step;
          const uint32_t lo = (uint32_t)key, hi = (uint32_t)(key >> 32);
          float v[8];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            v[t] = sT[((lo >> (8 * t)) & 0xFFu) * 32 + lane];
            v[4 + t] = sT[((hi >> (8 * t)) & 0xFFu) * 32 + lane];
          }
          uint4 w;
          w.x = __byte_perm(__float_as_uint(v[0]), __float_as_uint(v[1]), 0x7632);
          w.y = __byte_perm(__float_as_uint(v[2]), __float_as_uint(v[3]), 0x7632);
          w.z = __byte_perm(__float_as_uint(v[4]), __float_as_uint(v[5]), 0x7632);
          w.w = __byte_perm(__float_as_uint(v[6]), __float_as_uint(v[7]), 0x7632);
          *reinterpret_cast<uint4*>(sA + kmaj_off<S::KC>(r, 8 * q)) = w;
          if (with_b) {
            const float4 b0 = *reinterpret_cast<const float4*>(bc + 8 * q);
            const float4 b1 = *reinterpret_cast<const float4*>(bc + 8 * q + 4);
            bpart = fmaf(v[0], b0.x, bpart);
            bpart = fmaf(v[1], b0.y, bpart);
            bpart = fmaf(v[2], b0.z, bpart);
            bpart = fmaf(v[3], b0.w, bpart);
            bpart = fmaf(v[4], b1.x, bpart);
            bpart = fmaf(v[5], b1.y, bpart);
            bpart = fmaf(v[6], b1.z, bpart);
            bpart = fmaf(v[7], b1.w, bpart);
          }
        }
        if (with_b) {
          const float t = sb_hi + bpart;                            // TwoSum (Knuth)
          const float bb = t - sb_hi;
          sb_lo += (sb_hi - (t - bb)) + (bpart - bb);
          sb_hi = t;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (since == flush_every) {
        // chunks c - flush_every .. c - 1 are in D: wait for their MMAs, add D into
        // S; the MMA warp restarts D with chunk c only after every warp has arrived
        if (!__all_sync(0xffffffffu, u_wait(&gfree[gp.s], gp.ph))) {
          if (lane == 0) fail();
          break;
        }
        tmem_flush(false);
        since = 0;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(u_smem(&g_ready[sg])) : "memory");
      ++since;
      gp = g;
      g.next();
      t.next();
    }
  }
  __syncthreads();
  const int64_t issued = s_issued;
  if (!mma_warp && issued > 0 && !s_fail) {
    // the last issued chunk's commit tracks all earlier MMAs
    const int64_t cl = issued - 1;
    if (__all_sync(0xffffffffu, u_wait(&gfree[cl % GST], (uint32_t)((cl / GST) & 1)))) {
      if (issued == nchunks) tmem_flush(true);
    } else if (lane == 0) {
      fail();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && (s_fail || issued != nchunks)) atomicExch(err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr) : "memory");
}

static int gauss_kt(int terms) { return terms == 3 ? GShape<3>::KT : terms == 2 ? GShape<2>::KT : GShape<1>::KT; }
static size_t gauss_tile_bytes(int terms) {
  return terms == 3 ? GShape<3>::BStage : terms == 2 ? GShape<2>::BStage : GShape<1>::BStage;
}

// Launch shape of gauss_umma: row tiles of G x K splits x column tiles, one
// CTA per SM; K ranges in whole chunks of kt rows.
struct GaussGrid {
  int64_t mtiles, ntiles, ksplit, kchunk, nchunks;
};
static GaussGrid gauss_grid(int64_t m, int64_t n, int64_t d, int64_t kt) {
  GaussGrid g;
  g.mtiles = (d + kUG - 1) / kUG;
  g.ntiles = (n + kUN - 1) / kUN;
  g.ksplit = std::max<int64_t>(1, (int64_t)num_sms() / std::max<int64_t>(1, g.mtiles * g.ntiles));
  g.kchunk = (m + g.ksplit - 1) / g.ksplit;
  g.kchunk = ((g.kchunk + kt - 1) / kt) * kt;
  g.ksplit = (m + g.kchunk - 1) / g.kchunk;
  g.nchunks = (m + kt - 1) / kt;
  return g;
}
constexpr size_t kGaussTilesOffset = 8192 + 256;
constexpr int kGaussGroups = 32 * kUGenWarps / kUG;     // b-column partials per (K split, row)
// Workspace: the BF16 table (uploaded per call), the error word, the converted
// [A | b] tiles, then the per-K-split partial tiles of SA (d x n each) and of
// Sb (kGaussGroups x d each), sized for at most kSizingSms K splits per tile.
constexpr int64_t kSizingSms = 256;
static int64_t gauss_ksplit_bound(int64_t m, int64_t n, int64_t d, int64_t kt) {
  const int64_t tiles = ((d + kUG - 1) / kUG) * ((n + kUN - 1) / kUN);
  return std::max<int64_t>(1, std::min<int64_t>(kSizingSms / std::max<int64_t>(1, tiles), (m + kt - 1) / kt));
}
static size_t gauss_part_offset(int64_t m, int64_t n, int terms) {
  const int64_t kt = gauss_kt(terms);
  const int64_t nchunks = (m + kt - 1) / kt, ntiles = (n + kUN - 1) / kUN;
  return kGaussTilesOffset + (size_t)nchunks * ntiles * gauss_tile_bytes(terms);
}
size_t gauss_ws_bytes(int64_t m, int64_t n, int64_t d, int terms) {
  const size_t ks = (size_t)gauss_ksplit_bound(m, n, d, gauss_kt(terms));
  return gauss_part_offset(m, n, terms) + ks * (size_t)d * n * 4 + ks * kGaussGroups * (size_t)d * 4;
}

// SA and Sb as the sums of the K splits' partials, in split order (the result
// does not depend on the order in which the CTAs finished).
__global__ void __launch_bounds__(256)
gauss_reduce(const float* __restrict__ part, const float* __restrict__ partb, int64_t ksplit, int64_t d, int64_t n,
             float* __restrict__ SA, int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  const int64_t total = d * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total + d;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < total) {
      float acc = 0.f;
      for (int64_t y = 0; y < ksplit; ++y) acc += __ldg(part + y * total + e);
      SA[(e / n) * ldsa + e % n] = acc;
    } else {
      const int64_t row = e - total;
      float acc = 0.f;
      for (int64_t y = 0; y < ksplit * kGaussGroups; ++y) acc += __ldg(partb + y * d + row);
      Sb[row * sbs] = acc;
    }
  }
}

template <int T, int GS, int BS>
static sns_status gauss_launch(const uint8_t* tiles, const GaussGrid& gg, const DenseArgs& a, int64_t d, uint64_t s0,
                               const uint16_t* dtab, float scale, float* part, float* partb, int* err,
                               cudaStream_t st) {
  using S = GShape<T, GS, BS>;
  SNS_CUDA_TRY(raise_smem_limit((const void*)gauss_umma<T, GS, BS>));
  dim3 grid((unsigned)gg.mtiles, (unsigned)gg.ksplit, (unsigned)gg.ntiles);
  {
    SNS_PROF(K_GAUSS, st);
    gauss_umma<T, GS, BS><<<grid, 32 * (kUGenWarps + 1), S::Smem, st>>>(
        tiles, gg.ntiles, a.m, a.n, d, s0, dtab, gg.kchunk, scale, part, partb, err, S::Flush);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

template <int T>
static sns_status gauss_tensor(const DenseArgs& a, int64_t d, uint64_t s0, const uint16_t* dtab, float* SA,
                               int64_t ldsa, float* Sb, int64_t sbs, void* ws, int* err, cudaStream_t st) {
  using S = GShape<T>;
  const GaussGrid gg = gauss_grid(a.m, a.n, d, S::KT);
  uint8_t* tiles = static_cast<uint8_t*>(ws) + kGaussTilesOffset;
  {
    SNS_PROF(K_GAUSS, st);
    gauss_convert<T><<<num_sms() * 8, 256, 0, st>>>(static_cast<const float*>(a.A), a.lda,
                                                    static_cast<const float*>(a.b), a.m, a.n, gg.nchunks, gg.ntiles,
                                                    tiles);
  }
  SNS_LAUNCH_CHECK();
  if (gg.ksplit > gauss_ksplit_bound(a.m, a.n, d, S::KT)) return SNS_EINVAL;   // more SMs than the sizing bound
  const float scale = (float)(1.0 / std::sqrt((double)d));
  float* part = reinterpret_cast<float*>(static_cast<uint8_t*>(ws) + gauss_part_offset(a.m, a.n, T));
  float* partb = part + (size_t)gg.ksplit * d * a.n;
  const sns_status r = gauss_launch<T, S::GStages, S::BStages>(tiles, gg, a, d, s0, dtab, scale, part, partb, err, st);
  if (r != SNS_OK) return r;
  {
    SNS_PROF(K_GAUSS, st);
    gauss_reduce<<<num_sms() * 4, 256, 0, st>>>(part, partb, gg.ksplit, d, a.n, SA, ldsa, Sb, sbs);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

sns_status gauss_apply_dense(const DenseArgs& a, int64_t d, uint64_t seed, int terms, float* SA, int64_t ldsa,
                             float* Sb, int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (terms < 1 || terms > 3) return SNS_EINVAL;
  if (!ws || ws_bytes < gauss_ws_bytes(a.m, a.n, d, terms)) return SNS_ENOMEM;
  uint16_t* dtab = static_cast<uint16_t*>(ws);
  SNS_CUDA_TRY(cudaMemcpyAsync(dtab, table_host(), kGaussLevels * 2, cudaMemcpyHostToDevice, st));
  // SNSOLVE_GAUSS=simt selects the CUDA-core kernel (one BF16 term only)
  static int use_simt = -1;
  if (use_simt < 0) {
    const char* e = getenv("SNSOLVE_GAUSS");
    use_simt = (e && e[0] == 's') ? 1 : 0;
  }
  int* err = reinterpret_cast<int*>(static_cast<uint8_t*>(ws) + gauss_err_offset());
  SNS_CUDA_TRY(cudaMemsetAsync(err, 0, 4, st));
  const uint64_t s0 = shift_state(stream_state(seed, kStreamGaussian), (uint64_t)(a.row0 / 8) * (uint64_t)d);
  if (!use_simt || terms > 1) {
    switch (terms) {
      case 1: return gauss_tensor<1>(a, d, s0, dtab, SA, ldsa, Sb, sbs, ws, err, st);
      case 2: return gauss_tensor<2>(a, d, s0, dtab, SA, ldsa, Sb, sbs, ws, err, st);
      default: return gauss_tensor<3>(a, d, s0, dtab, SA, ldsa, Sb, sbs, ws, err, st);
    }
  }
  // the SIMT kernel adds into SA and Sb
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
    gauss_simt<<<grid, 256, 0, st>>>(static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b), a.m, a.n,
                                     d, s0, dtab, kchunk, (float)(1.0 / std::sqrt((double)d)), SA, ldsa, Sb, sbs);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

}  // namespace sns
