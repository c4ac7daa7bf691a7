// CountSketch apply, deterministic variant, bulk-copy pipeline (dense FP32).
//
// Phase 1 (countsketch.cu) counting-sorts the row ids of every 4096-row block by
// bucket.  Phase 1b here turns those per-block runs into one bucket-major list
// (rows of bucket 0 in ascending order, then bucket 1, ...).  Phase 2 splits
// every bucket's rows into P contiguous parts; a work item is (bucket, part,
// column tile).  In each CTA one producer warp walks its items, reads the
// item's row ids and b entries with coalesced loads, and issues one
// cp.async.bulk copy per row (the row's columns of the tile, 1 KB at n = 256)
// into a shared-memory ring owned by consumer warp (j mod 8), j being the row's
// position in the item.  Consumer warps wait on the slot's mbarrier, add the
// signed row into register accumulators (two per warp, alternating rows), and
// free the slot.  At the end of an item the 16 partial rows are added in a
// fixed tree order; parts of a bucket are added in part order by the last CTA
// to finish the bucket.  The summation order depends only on (m, d, n, P), not
// on the grid, so results are bitwise reproducible.
//
// All mbarrier waits are bounded; a wait that gives up raises a CTA-wide abort
// flag (every later wait returns at once), records an error word, and the
// producer waits (bounded) for its last copy before the CTA exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace sns {

constexpr int kTmaWC = 8;          // consumer warps
constexpr int kTmaCH = 512;        // producer row-list chunk
constexpr uint32_t kEnd = 0xFFFFFFFFu;
constexpr long long kWaitLimit = 1LL << 22;
constexpr int kListRowsPerBlock = 4096;   // phase-1 block height (matches countsketch.cu)
constexpr int kChunkRows = 128;           // rows per warp work item of the warp gather

template <int CT>
struct TmaCfg {
  static constexpr int SW = CT == 256 ? 6 : 8;   // slots per consumer ring
  static constexpr int NS = kTmaWC * SW;
  static constexpr size_t smem_bytes() {
    return (size_t)NS * CT * 4                    // slots
           + (size_t)2 * kTmaWC * 2 * (CT + 1) * 4  // partial rows, double-buffered
           + (size_t)kTmaCH * 8                   // row ids + b values
           + (size_t)NS * 8                       // meta
           + (size_t)NS * 16;                     // full + empty barriers
  }
};

SNS_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
SNS_D void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
SNS_D void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
SNS_D void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
SNS_D bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; gives up early when the CTA is aborting.
SNS_D bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  for (long long i = 0; i < kWaitLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && *abort) return false;
  }
  if (abort) *abort = 1;
  return false;
}
SNS_D void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
SNS_D void consumer_bar() { asm volatile("bar.sync 1, %0;" ::"r"(kTmaWC * 32) : "memory"); }

// ---------------------------------------------------------------------------
// Phase 1b: bucket bases (exclusive scan of the bucket totals, done by every
// CTA in shared memory) and the bucket-major row list.  One warp per bucket.
__global__ void __launch_bounds__(256)
cs_build_list(uint32_t d, int64_t nblk, const uint32_t* __restrict__ sorted, const uint32_t* __restrict__ seg,
              const uint32_t* __restrict__ btot, uint32_t* __restrict__ bbase, uint32_t* __restrict__ list,
              uint32_t* __restrict__ cbase, uint32_t* __restrict__ ctab, float* __restrict__ SA, int64_t ldsa,
              float* __restrict__ Sb, int64_t sbs, int64_t n) {
  extern __shared__ uint32_t sbase[];   // d bucket bases, then d chunk bases
  uint32_t* scb = sbase + d;
  __shared__ uint32_t wsum[8], wsum2[8];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = ((int)d + 255) / 256;
  const int k0 = tid * per, k1 = min((int)d, k0 + per);
  uint32_t local = 0, lch = 0;
  for (int k = k0; k < k1; ++k) {
    local += btot[k];
    lch += (btot[k] + kChunkRows - 1) / kChunkRows;
  }
  uint32_t incl = local, inc2 = lch;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    const uint32_t t2 = __shfl_up_sync(0xffffffffu, inc2, o);
    if (lane >= o) { incl += t; inc2 += t2; }
  }
  if (lane == 31) { wsum[w] = incl; wsum2[w] = inc2; }
  __syncthreads();
  uint32_t run = incl - local, run2 = inc2 - lch;
  for (int ww = 0; ww < w; ++ww) { run += wsum[ww]; run2 += wsum2[ww]; }
  for (int k = k0; k < k1; ++k) {
    sbase[k] = run;
    scb[k] = run2;
    if (blockIdx.x == 0) { bbase[k] = run; cbase[k] = run2; }
    run += btot[k];
    run2 += (btot[k] + kChunkRows - 1) / kChunkRows;
  }
  __syncthreads();
  if (blockIdx.x == 0 && tid == blockDim.x - 1) cbase[d] = run2;       // total chunk count
  for (int64_t k = (int64_t)blockIdx.x * 8 + w; k < d; k += (int64_t)gridDim.x * 8) {
    const uint32_t nch = (btot[k] + kChunkRows - 1) / kChunkRows;
    for (uint32_t c = lane; c < nch; c += 32) ctab[scb[k] + c] = (uint32_t)k;
    if (SA && btot[k] == 0) {
      // a bucket no row hashed to has no work item in phase 2: its rows are zero
      for (int64_t c = lane; c < n; c += 32) SA[k * ldsa + c] = 0.f;
      if (lane == 0) Sb[k * sbs] = 0.f;
    }
    uint32_t pos = sbase[k];
    // segment words of up to kSegAhead rounds of 32 blocks load together, and
    // each segment's rows are copied 8 at a time, so a bucket costs a few
    // dependent memory round trips instead of two per round
    constexpr int kSegAhead = 8;
    for (int64_t bb = 0; bb < nblk; bb += 32 * kSegAhead) {
      uint32_t sv[kSegAhead];
#pragma unroll
      for (int r = 0; r < kSegAhead; ++r) {
        const int64_t blk = bb + r * 32 + lane;
        sv[r] = blk < nblk ? __ldg(seg + (size_t)k * nblk + blk) : 0u;
      }
#pragma unroll
      for (int r = 0; r < kSegAhead; ++r) {
        const int64_t blk = bb + r * 32 + lane;
        const uint32_t c = sv[r] & 0xFFFFu, st = sv[r] >> 16;
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += t;
        }
        const uint32_t ex = inc - c;
        const uint32_t* src = sorted + blk * kListRowsPerBlock + st;
        uint32_t* dst = list + pos + ex;
        for (uint32_t i0 = 0; i0 < c; i0 += 8) {
          uint32_t v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = (i0 + u < c) ? __ldg(src + i0 + u) : 0u;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (i0 + u < c) dst[i0 + u] = v[u];
        }
        pos += __shfl_sync(0xffffffffu, inc, 31);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Phases 1 + 1b in one cooperative launch (one CTA per block of rows_per_blk
// = 4096 consecutive rows, all co-resident; measured: 16 warps and two CTAs
// per SM ran faster than one 32-warp CTA per SM with equal blocks): the same hash, per-warp histograms and stable per-block order
// as cs_sort_blocks, and the same bucket-major list, chunk tables and
// empty-bucket zeroing as cs_build_list, without the intermediate per-block
// sorted array.  Two grid barriers separate the phases:
//   A  per block: hash every row once (bucket | sign kept in shared memory),
//      per-warp bucket histograms and each row's stable rank among the rows
//      of its bucket that its warp hashed before it, block totals ->
//      seg[k * nblk + blk];
//   B  per bucket (buckets spread over the CTAs): exclusive scan of its block
//      totals in block order (the bucket's start in each block), total -> btot;
//   C  per CTA: bucket bases and chunk bases by scanning btot (each CTA scans
//      all d totals itself; btot and the block's starts are read in one
//      round trip), chunk table and zeroed SA rows for its buckets, then its
//      block's rows scattered to list[bbase + block start + warp offset +
//      rank] (no second multisplit), rows of a bucket in ascending order.
// The grid barriers are bounded: a CTA whose wait gives up sets the error word
// and skips its remaining work but still arrives at later barriers; every CTA
// reads the word before scattering, positions are checked against m, and the
// gather returns at once when the word is set.
constexpr int kPlanWarps = 16;
SNS_D uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
SNS_D int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Arrival counter `bar` grows monotonically; barrier number e waits for (e + 1) * G
// arrivals.  Returns, identically in every thread of the CTA, whether the error
// word was clear after the wait (one read by thread 0, broadcast through shared
// memory, so the CTA's control flow stays uniform).
SNS_D bool grid_barrier(uint32_t* bar, uint32_t target, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    bool ok = false;
    for (long long it = 0; it < kWaitLimit; ++it) {
      if (ld_acquire_u32(bar) >= target) {
        ok = true;
        break;
      }
      if (it >= 64) __nanosleep(64);
    }
    if (!ok) atomicExch(err, 1);
    __threadfence();
    s_ok = (ok && ld_acquire_i32(err) == 0) ? 1 : 0;
  }
  __syncthreads();
  return s_ok != 0;
}
// Exclusive scan over k < d of f(k) into out[k] (shared memory), every thread
// owning a contiguous run of ceil(d / 256) buckets; returns the total.
template <typename F>
SNS_D uint32_t block_scan_buckets(uint32_t d, F&& f, uint32_t* out, uint32_t* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = ((int)d + blockDim.x - 1) / blockDim.x;
  const int k0 = tid * per, k1 = min((int)d, k0 + per);
  uint32_t local = 0;
  for (int k = k0; k < k1; ++k) local += f(k);
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();                       // wsum free (an earlier scan may still read it)
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  uint32_t run = incl - local, total = 0;
  for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
    if (ww < w) run += wsum[ww];
    total += wsum[ww];
  }
  for (int k = k0; k < k1; ++k) {
    out[k] = run;
    run += f(k);
  }
  __syncthreads();
  return total;
}

// Lanes of the warp holding the same value v (< 2^nbits) as this lane: one
// ballot per bit, the same mask __match_any_sync returns (warp multisplit).
SNS_D unsigned equal_lanes(uint32_t v, int nbits) {
  unsigned peers = 0xffffffffu;
  for (int bit = 0; bit < nbits; ++bit) {
    const bool set = (v >> bit) & 1u;
    const unsigned bal = __ballot_sync(0xffffffffu, set);
    peers &= set ? bal : ~bal;
  }
  return peers;
}

__global__ void __launch_bounds__(kPlanWarps * 32)
cs_plan_coop(int64_t m, uint32_t d, uint64_t s0, int64_t nblk, uint32_t* __restrict__ seg,
             uint32_t* __restrict__ ticket, int64_t nticket, uint32_t* __restrict__ btot, uint32_t* __restrict__ bbase,
             uint32_t* __restrict__ list, uint32_t* __restrict__ cbase, uint32_t* __restrict__ ctab,
             float* __restrict__ SA, int64_t ldsa, float* __restrict__ Sb, int64_t sbs, int64_t n,
             uint32_t* __restrict__ bar, int* __restrict__ err, int nbits, int rows_per_blk) {
  extern __shared__ __align__(16) uint8_t psm[];
  uint16_t* cnt = reinterpret_cast<uint16_t*>(psm);                 // [W][d] per-warp counts, then offsets
  uint16_t* hb = cnt + (size_t)kPlanWarps * d;                       // [R] bucket | sign << 15
  uint16_t* rk = hb + rows_per_blk;                                  // [R] rank within (warp, bucket)
  uint32_t* sb = reinterpret_cast<uint32_t*>(rk + rows_per_blk);     // [d] bases; then [d] totals, [d] starts (C)
  __shared__ uint32_t wsum[kPlanWarps];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t blk = blockIdx.x;
  const int64_t r0 = blk * rows_per_blk;
  const uint32_t G = gridDim.x;
  const int kRowsPerWarp = rows_per_blk / kPlanWarps;                // a multiple of 32
  constexpr uint32_t kNone = 0xFFFFu;
  const uint32_t kOut = (1u << nbits) - 1u;        // >= d: groups the rows past m in the masks
  // a block with no row past m needs no bit for kOut
  const int nb = (r0 + rows_per_blk <= m && nbits > 1 && ((d - 1) >> (nbits - 1)) == 0) ? nbits - 1 : nbits;

  // ---- A: hash, per-warp histograms, block totals
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + tid; i < nticket; i += (int64_t)G * blockDim.x) ticket[i] = 0;
  if ((d & 7) == 0) {
    uint4* c4 = reinterpret_cast<uint4*>(cnt);
    for (int i = tid; i < kPlanWarps * (int)d / 8; i += blockDim.x) c4[i] = make_uint4(0u, 0u, 0u, 0u);
  } else {
    for (int i = tid; i < kPlanWarps * (int)d; i += blockDim.x) cnt[i] = 0;
  }
  __syncthreads();
  for (int j = 0; j < kRowsPerWarp; j += 32) {
    const int loc = w * kRowsPerWarp + j + lane;
    const int64_t row = r0 + loc;
    uint32_t h = kNone, sgn = 0;
    if (row < m) {
      const uint64_t key = splitmix_at(s0, (uint64_t)row);
      h = bucket_of(key, d);
      sgn = (uint32_t)(key >> 63);
    }
    hb[loc] = (uint16_t)(h == kNone ? kNone : (h | (sgn << 15)));
    const unsigned peers = equal_lanes(h == kNone ? kOut : h, nb);
    const uint32_t before = h != kNone ? cnt[w * d + h] : 0u;   // every peer reads it before the update
    rk[loc] = (uint16_t)(before + __popc(peers & ((1u << lane) - 1u)));
    __syncwarp();
    if (h != kNone && lane == __ffs(peers) - 1) cnt[w * d + h] = (uint16_t)(before + __popc(peers));
    __syncwarp();
  }
  __syncthreads();
  // block totals; per-warp counts become offsets within the block's bucket run
  for (int k = tid; k < (int)d; k += blockDim.x) {
    uint32_t tot = 0;
    for (int ww = 0; ww < kPlanWarps; ++ww) {
      const uint32_t c = cnt[ww * d + k];
      cnt[ww * d + k] = (uint16_t)tot;
      tot += c;
    }
    seg[(size_t)k * nblk + blk] = tot;
  }
  const bool ok1 = grid_barrier(bar, G, err);

  // ---- B: per bucket, exclusive scan of the block totals; bucket totals
  // (the block totals of 8 rounds of 32 blocks are loaded at once)
  if (ok1) {
    constexpr int kAhead = 8;
    for (int64_t k = (int64_t)w * G + blockIdx.x; k < d; k += (int64_t)G * kPlanWarps) {
      uint32_t* sk = seg + (size_t)k * nblk;
      uint32_t run = 0;
      for (int64_t b0 = 0; b0 < nblk; b0 += 32 * kAhead) {
        uint32_t cv[kAhead];
#pragma unroll
        for (int r = 0; r < kAhead; ++r) {
          const int64_t b = b0 + r * 32 + lane;
          cv[r] = b < nblk ? __ldcg(sk + b) : 0u;
        }
#pragma unroll
        for (int r = 0; r < kAhead; ++r) {
          const int64_t b = b0 + r * 32 + lane;
          const uint32_t c = cv[r];
          uint32_t incl = c;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
          }
          if (b < nblk) sk[b] = run + incl - c;
          run += __shfl_sync(0xffffffffu, incl, 31);
        }
      }
      if (lane == 0) btot[k] = run;
    }
  }
  if (!grid_barrier(bar, 2 * G, err)) return;           // CTA-uniform

  // ---- C: bases, chunk tables, empty buckets, scatter.  The bucket totals
  // and this block's starts are read from L2 together, into shared memory.
  uint32_t* stot = sb + d;
  uint32_t* sst = sb + 2 * (size_t)d;
  for (int k = tid; k < (int)d; k += blockDim.x) {
    stot[k] = __ldcg(btot + k);
    sst[k] = __ldcg(seg + (size_t)k * nblk + blk);
  }
  __syncthreads();
  const uint32_t nchunks =
      block_scan_buckets(d, [&](int k) { return (stot[k] + kChunkRows - 1) / kChunkRows; }, sb, wsum);
  if (blockIdx.x == 0 && tid == 0) cbase[d] = nchunks;
  for (int64_t k = (int64_t)w * G + blockIdx.x; k < d; k += (int64_t)G * kPlanWarps) {
    const uint32_t len = stot[k];
    const uint32_t nch = (len + kChunkRows - 1) / kChunkRows;
    for (uint32_t c = lane; c < nch; c += 32) ctab[sb[k] + c] = (uint32_t)k;
    if (lane == 0) cbase[k] = sb[k];
    if (len == 0) {
      // a bucket no row hashed to has no gather item: its rows are zero
      for (int64_t c = lane; c < n; c += 32) SA[k * ldsa + c] = 0.f;
      if (lane == 0) Sb[k * sbs] = 0.f;
    }
  }
  block_scan_buckets(d, [&](int k) { return stot[k]; }, sb, wsum);
  for (int k = tid; k < (int)d; k += blockDim.x) {
    if (blockIdx.x == 0) bbase[k] = sb[k];
    sb[k] += sst[k];                                          // this block's start in bucket k
  }
  // the gather may be scheduled now; it waits for this grid to complete
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __syncthreads();
  for (int j = 0; j < kRowsPerWarp; j += 32) {
    const int loc = w * kRowsPerWarp + j + lane;
    const uint32_t hw = hb[loc];
    if (hw != kNone) {
      const uint32_t h = hw & 0x7FFFu;
      const uint32_t pos = sb[h] + cnt[w * d + h] + rk[loc];
      if (pos < (uint64_t)m) list[pos] = (uint32_t)(r0 + loc) | ((hw >> 15) << 31);
    }
  }
}

size_t cs_plan_smem(int64_t d, int64_t rows_per_blk) {
  return (size_t)kPlanWarps * d * 2 + (size_t)rows_per_blk * 4 + (size_t)d * 12;
}

// ---------------------------------------------------------------------------
template <int CT>
__global__ void __launch_bounds__((kTmaWC + 1) * 32)
cs_gather_tma(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t n, uint32_t d,
              int64_t P, int64_t ntile, const uint32_t* __restrict__ list, const uint32_t* __restrict__ btot,
              const uint32_t* __restrict__ bbase, uint32_t* __restrict__ ticket, float* __restrict__ part_buf,
              float* __restrict__ SA, int64_t ldsa, float* __restrict__ Sb, int64_t sbs, int* __restrict__ err) {
  using Cfg = TmaCfg<CT>;
  constexpr int WC = kTmaWC, SW = Cfg::SW, NS = Cfg::NS, CH = kTmaCH, NCH = CT / 128;
  extern __shared__ __align__(128) uint8_t sm[];
  float* slots = reinterpret_cast<float*>(sm);
  float* red = slots + (size_t)NS * CT;
  uint32_t* rl = reinterpret_cast<uint32_t*>(red + (size_t)2 * WC * 2 * (CT + 1));
  float* bl = reinterpret_cast<float*>(rl + CH);
  uint2* meta = reinterpret_cast<uint2*>(bl + CH);
  uint64_t* full = reinterpret_cast<uint64_t*>(meta + NS);
  uint64_t* empty = full + NS;
  __shared__ volatile int s_abort;
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t nitems = (int64_t)d * P * ntile;

  if (w == WC) {
    // ------------------------------------------------------------ producer
    uint32_t cnt = 0;            // lane l < WC: slots used so far in ring l
    int last_slot = -1;
    uint32_t last_par = 0;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
      if (__any_sync(0xffffffffu, s_abort != 0)) break;
      const int64_t t = item % ntile, kp = item / ntile, p = kp % P, k = kp / P;
      const int64_t col0 = t * CT;
      const uint32_t bytes = (uint32_t)(min((int64_t)CT, n - col0) * 4);
      const int64_t len = btot[k], base = bbase[k];
      const int64_t lo = base + len * p / P, hi = base + len * (p + 1) / P;
      const int64_t J = hi - lo;
      for (int64_t c0 = 0; c0 < J; c0 += CH) {
        if (__any_sync(0xffffffffu, s_abort != 0)) break;
        const int nrow = (int)min((int64_t)CH, J - c0);
        for (int r = lane; r < nrow; r += 32) rl[r] = __ldg(list + lo + c0 + r);
        __syncwarp();
        for (int r = lane; r < nrow; r += 32) bl[r] = __ldg(b + (rl[r] & 0x7FFFFFFFu));
        __syncwarp();
        for (int r0 = 0; r0 < nrow; r0 += 32) {
          const int r = r0 + lane;
          const int64_t jj = c0 + r;
          const int ww = (int)(jj % WC);
          const uint32_t kth = (uint32_t)(jj / WC);
          const uint32_t cw = __shfl_sync(0xffffffffu, cnt, ww);
          if (r < nrow && !s_abort) {
            const uint32_t pos = cw + kth;
            const int slot = ww * SW + (int)(pos % SW);
            const uint32_t par = (pos / SW) & 1u;
            if (mbar_wait(empty + slot, par ^ 1u, &s_abort)) {
              const uint32_t rid = rl[r];
              meta[slot] = make_uint2(rid, __float_as_uint(bl[r]));
              mbar_arrive_expect_tx(full + slot, bytes);
              bulk_g2s(slots + (size_t)slot * CT, A + (int64_t)(rid & 0x7FFFFFFFu) * lda + col0, bytes, full + slot);
              last_slot = slot;
              last_par = par;
            }
          }
        }
        __syncwarp();
      }
      // end-of-item markers, one per consumer ring
      if (lane < WC && !s_abort) {
        const uint32_t nl = (J > lane) ? (uint32_t)((J - lane + WC - 1) / WC) : 0u;
        const uint32_t pos = cnt + nl;
        const int slot = lane * SW + (int)(pos % SW);
        const uint32_t par = (pos / SW) & 1u;
        if (mbar_wait(empty + slot, par ^ 1u, &s_abort)) {
          meta[slot] = make_uint2(kEnd, 0u);
          mbar_arrive(full + slot);
        }
        cnt = pos + 1;
      }
      __syncwarp();
    }
    if (__any_sync(0xffffffffu, s_abort != 0)) {
      if (lane == 0) atomicExch(err, 1);
      if (last_slot >= 0) mbar_wait(full + last_slot, last_par, nullptr);   // own copy lands before exit
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  uint32_t pos = 0;
  int it = 0;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
    const int64_t t = item % ntile, kp = item / ntile, p = kp % P, k = kp / P;
    const int64_t col0 = t * CT;
    float acc[2][NCH][4];
    float accb[2] = {0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[a][q][v] = 0.f;
    uint32_t kth = 0;
    for (;;) {
      if (__any_sync(0xffffffffu, s_abort != 0)) break;
      const int slot = w * SW + (int)(pos % SW);
      const uint32_t par = (pos / SW) & 1u;
      const bool got = mbar_wait(full + slot, par, &s_abort);
      if (!__all_sync(0xffffffffu, got)) break;
      const uint2 mt = meta[slot];
      if (mt.x == kEnd) {
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + slot);
        ++pos;
        break;
      }
      const float* row = slots + (size_t)slot * CT;
      float4 v[NCH];
#pragma unroll
      for (int q = 0; q < NCH; ++q) v[q] = *reinterpret_cast<const float4*>(row + q * 128 + lane * 4);
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + slot);
      const bool neg = (mt.x >> 31) != 0;
      const float bv = __uint_as_float(mt.y);
      // two accumulators, alternating rows (warp-uniform branch keeps them in registers)
      if (kth & 1) {
#pragma unroll
        for (int q = 0; q < NCH; ++q) {
          acc[1][q][0] += neg ? -v[q].x : v[q].x;
          acc[1][q][1] += neg ? -v[q].y : v[q].y;
          acc[1][q][2] += neg ? -v[q].z : v[q].z;
          acc[1][q][3] += neg ? -v[q].w : v[q].w;
        }
        accb[1] += neg ? -bv : bv;
      } else {
#pragma unroll
        for (int q = 0; q < NCH; ++q) {
          acc[0][q][0] += neg ? -v[q].x : v[q].x;
          acc[0][q][1] += neg ? -v[q].y : v[q].y;
          acc[0][q][2] += neg ? -v[q].z : v[q].z;
          acc[0][q][3] += neg ? -v[q].w : v[q].w;
        }
        accb[0] += neg ? -bv : bv;
      }
      ++kth;
      ++pos;
    }
    // partial rows of this warp
    float* rb = red + (size_t)(it & 1) * WC * 2 * (CT + 1);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      float* rr = rb + (size_t)(w * 2 + a) * (CT + 1);
#pragma unroll
      for (int q = 0; q < NCH; ++q) {
        rr[q * 128 + lane * 4 + 0] = acc[a][q][0];
        rr[q * 128 + lane * 4 + 1] = acc[a][q][1];
        rr[q * 128 + lane * 4 + 2] = acc[a][q][2];
        rr[q * 128 + lane * 4 + 3] = acc[a][q][3];
      }
      if (lane == 0) rr[CT] = accb[a];
    }
    consumer_bar();
    // On abort every consumer still runs the same barrier sequence; only the
    // stores are skipped.
    const bool ab = s_abort != 0;
    // fixed-order tree over the 2*WC partial rows
    const int ctid = threadIdx.x;  // 0 .. WC*32-1
    float* pb = part_buf + ((size_t)(k * ntile + t) * P + p) * (CT + 1);
    for (int c = ctid; c <= CT; c += WC * 32) {
      float vals[2 * WC];
#pragma unroll
      for (int i = 0; i < 2 * WC; ++i) vals[i] = rb[(size_t)i * (CT + 1) + c];
#pragma unroll
      for (int s = WC; s > 0; s >>= 1)
#pragma unroll
        for (int i = 0; i < s; ++i) vals[i] += vals[i + s];
      if (ab) continue;
      if (P > 1) {
        pb[c] = vals[0];
      } else if (c < CT) {
        if (col0 + c < n) SA[k * ldsa + col0 + c] = vals[0];
      } else if (t == 0) {
        Sb[k * sbs] = vals[0];
      }
    }
    if (P > 1) {
      __threadfence();
      consumer_bar();
      if (ctid == 0) s_last = (!s_abort && atomicAdd(ticket + k * ntile + t, 1u) == (uint32_t)(P - 1)) ? 1 : 0;
      consumer_bar();
      if (s_last) {
        __threadfence();
        const float* pk = part_buf + (size_t)(k * ntile + t) * P * (CT + 1);
        for (int c = ctid; c <= CT; c += WC * 32) {
          float s = 0.f;
          for (int64_t pp = 0; pp < P; ++pp) s += __ldcg(pk + pp * (CT + 1) + c);
          if (c < CT) {
            if (col0 + c < n) SA[k * ldsa + col0 + c] = s;
          } else if (t == 0) {
            Sb[k * sbs] = s;
          }
        }
      }
    }
  }
}


// ---------------------------------------------------------------------------
// Phase 2, warp variant: a warp item is (chunk of kChunkRows consecutive
// entries of one bucket's list, column tile of kWarpCT = 128 columns, i.e.
// 512 B of each row).  Warps fetch items from a global counter, one item
// ahead: the next item's index and metadata load while the current item
// streams.  The warp loads the chunk's row ids 32 at a time (one coalesced
// load; the next 32 load while the current rows stream), keeps 8 row tiles in
// flight (one float4 per lane each), and adds them into two register
// accumulators (even / odd rows).  b entries are added per lane and summed by a
// fixed shuffle tree.  The chunk's row goes to the partial buffer; the last
// warp to finish a (bucket, tile) (ticket) adds the bucket's chunk rows in
// chunk order.  A bucket with one chunk is written directly.  Which warp runs
// an item does not change its arithmetic, so results are deterministic.
// VPL float4 per lane per row (column tile CT = 128 VPL: 512 B or whole 1 KB
// rows at n = 256), U rows in flight per warp.
constexpr int kWarpCT = 128;
template <int VPL, int U>
__global__ void __launch_bounds__(256, VPL == 1 ? 3 : 2)
cs_gather_warp(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t n, int64_t ntile,
               const uint32_t* __restrict__ list, const uint32_t* __restrict__ btot,
               const uint32_t* __restrict__ bbase, const uint32_t* __restrict__ cbase,
               const uint32_t* __restrict__ ctab, uint32_t d, uint32_t* __restrict__ ticket,
               uint32_t* __restrict__ next_item, float* __restrict__ part, float* __restrict__ SA, int64_t ldsa,
               float* __restrict__ Sb, int64_t sbs, const int* __restrict__ err) {
  // launched as a programmatic dependent of the plan kernel: nothing the plan
  // writes is read before the plan grid has completed (no-op otherwise)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // a plan phase that gave up a bounded wait left its tables incomplete
  if (*err != 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = cbase[d];
  const int64_t nitems = nchunks * ntile;
  // item metadata: (bucket, first and end list entry); the next item's index
  // and metadata are fetched while the current item streams its rows
  struct Item {
    int64_t g, lo, hi, len;
    uint32_t k;
  };
  auto fetch = [&]() {
    uint32_t gi = 0;
    if (lane == 0) gi = atomicAdd(next_item, 1u);
    Item it;
    it.g = __shfl_sync(0xffffffffu, gi, 0);
    it.k = 0;
    it.lo = it.hi = it.len = 0;
    if (it.g < nitems) {
      const int64_t chunk = it.g / ntile;
      it.k = __ldg(ctab + chunk);
      const int64_t c = chunk - __ldg(cbase + it.k);
      it.len = __ldg(btot + it.k);
      const int64_t base = __ldg(bbase + it.k);
      it.lo = base + c * kChunkRows;
      it.hi = min(base + it.len, it.lo + kChunkRows);
    }
    return it;
  };
  Item cur = fetch();
  while (cur.g < nitems) {
    const Item nxt = fetch();
    const int64_t g = cur.g, t = g % ntile;
    const uint32_t k = cur.k;
    const int64_t len = cur.len, lo = cur.lo, hi = cur.hi;
    constexpr int CT = 128 * VPL;
    const int64_t col0 = t * CT;
    bool okc[VPL];
    float4 a0[VPL], e0[VPL];                                 // even / odd rows
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      okc[v] = col0 + v * 128 + lane * 4 < n;
      a0[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      e0[v] = a0[v];
    }
    float accb = 0.f;
    uint32_t rid_next = (lo + lane < hi) ? __ldg(list + lo + lane) : 0u;
    for (int64_t j0 = lo; j0 < hi; j0 += 32) {
      const int nr = (int)min((int64_t)32, hi - j0);
      const uint32_t rid_l = rid_next;
      // the next 32 row ids load while these rows stream
      rid_next = (j0 + 32 + lane < hi) ? __ldg(list + j0 + 32 + lane) : 0u;
      if (t == 0 && lane < nr) {
        const float bv = __ldg(b + (rid_l & 0x7FFFFFFFu));
        accb += (rid_l >> 31) ? -bv : bv;
      }
      for (int r = 0; r < nr; r += U) {
        float4 x[U][VPL];
        uint32_t rid[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          rid[u] = __shfl_sync(0xffffffffu, rid_l, (r + u) & 31);
          const float* rp = A + (int64_t)(rid[u] & 0x7FFFFFFFu) * lda + col0 + lane * 4;
#pragma unroll
          for (int v = 0; v < VPL; ++v) {
            const bool ok = ((r + u) < nr) && okc[v];
            x[u][v] = ok ? __ldg(reinterpret_cast<const float4*>(rp + v * 128)) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float sg = (rid[u] >> 31) ? -1.f : 1.f;
#pragma unroll
          for (int v = 0; v < VPL; ++v) {
            float4& p0 = (u & 1) ? e0[v] : a0[v];
            p0.x = fmaf(sg, x[u][v].x, p0.x);
            p0.y = fmaf(sg, x[u][v].y, p0.y);
            p0.z = fmaf(sg, x[u][v].z, p0.z);
            p0.w = fmaf(sg, x[u][v].w, p0.w);
          }
        }
      }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      a0[v].x += e0[v].x; a0[v].y += e0[v].y; a0[v].z += e0[v].z; a0[v].w += e0[v].w;
    }
    accb = warp_sum(accb);
    const int64_t nch_k = (len + kChunkRows - 1) / kChunkRows;
    if (nch_k == 1) {
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        float* out = SA + (int64_t)k * ldsa + col0 + v * 128 + lane * 4;
        if (okc[v]) { out[0] = a0[v].x; out[1] = a0[v].y; out[2] = a0[v].z; out[3] = a0[v].w; }
      }
      if (t == 0 && lane == 0) Sb[(int64_t)k * sbs] = accb;
      cur = nxt;
      continue;
    }
    float* pr = part + (size_t)g * (CT + 4);
#pragma unroll
    for (int v = 0; v < VPL; ++v) reinterpret_cast<float4*>(pr)[v * 32 + lane] = a0[v];
    if (lane == 0) pr[CT] = accb;
    __threadfence();
    __syncwarp();
    uint32_t old = 0;
    if (lane == 0) old = atomicAdd(ticket + (int64_t)k * ntile + t, 1u);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != (uint32_t)(nch_k - 1)) {
      cur = nxt;
      continue;
    }
    __threadfence();
    // last warp of bucket k, tile t: add the chunk rows in chunk order
    const int64_t g0 = (int64_t)__ldg(cbase + k) * ntile + t;
    float4 s0[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) s0[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    float sb = 0.f;
    for (int64_t q = 0; q < nch_k; ++q) {
      const float* pq = part + (size_t)(g0 + q * ntile) * (CT + 4);
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const float4 v0 = __ldcg(reinterpret_cast<const float4*>(pq) + v * 32 + lane);
        s0[v].x += v0.x; s0[v].y += v0.y; s0[v].z += v0.z; s0[v].w += v0.w;
      }
      sb += __ldcg(pq + CT);
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      float* out = SA + (int64_t)k * ldsa + col0 + v * 128 + lane * 4;
      if (okc[v]) { out[0] = s0[v].x; out[1] = s0[v].y; out[2] = s0[v].z; out[3] = s0[v].w; }
    }
    if (t == 0 && lane == 0) Sb[(int64_t)k * sbs] = sb;
    cur = nxt;
  }
}

int64_t cs_warp_max_chunks(int64_t m, int64_t d) { return (m + kChunkRows - 1) / kChunkRows + d; }
// ---------------------------------------------------------------------------
int64_t cs_tma_parts(int64_t m, int64_t d) {
  const int64_t per = d * 256;
  int64_t P = (m + per / 2) / per;
  return P < 1 ? 1 : P;
}

bool cs_tma_eligible(const DenseArgs& a) {
  return !a.f64 && a.n % 4 == 0 && a.lda % 4 == 0 && ((uintptr_t)a.A % 16) == 0 && a.n >= 32;
}

template <int CT>
static sns_status launch_tma(const DenseArgs& a, int64_t d, const CsLayout& L, uint8_t* ws, float* SA, int64_t ldsa,
                             float* Sb, int64_t sbs, cudaStream_t st) {
  const size_t smem = TmaCfg<CT>::smem_bytes();
  auto kern = cs_gather_tma<CT>;
  SNS_CUDA_TRY(raise_smem_limit((const void*)kern));
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (kTmaWC + 1) * 32, smem));
  if (occ < 1) occ = 1;
  const int64_t ntile = (a.n + CT - 1) / CT;
  const int64_t items = d * L.tma_parts * ntile;
  const int64_t grid = std::min<int64_t>(items, (int64_t)num_sms() * occ);
  {
    SNS_PROF(K_CS_GATHER, st);
    kern<<<(unsigned)grid, (kTmaWC + 1) * 32, smem, st>>>(
        static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b), a.n, (uint32_t)d, L.tma_parts, ntile,
        reinterpret_cast<const uint32_t*>(ws + L.off_list), reinterpret_cast<const uint32_t*>(ws + L.off_btot),
        reinterpret_cast<const uint32_t*>(ws + L.off_bbase), reinterpret_cast<uint32_t*>(ws + L.off_ticket),
        reinterpret_cast<float*>(ws + L.off_part), SA, ldsa, Sb, sbs, reinterpret_cast<int*>(ws + L.off_err));
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

// Column tile of the warp gather: 1 = 512-byte half rows (128 columns), 2 =
// whole 1 KB rows (256 columns) per work item.  Default: whole rows when n > 128
// (measured at 2^20 x 256: gather 0.177 ms vs 0.184 ms with half rows, 0.186 ms
// with whole rows and 4 rows in flight); SNSOLVE_CS_WARP_TILE=128|256|256u4
// overrides it.
static int warp_tile_choice() {
  static const int sel = [] {
    const char* e = getenv("SNSOLVE_CS_WARP_TILE");
    if (!e) return 0;
    if (e[0] == '2' && e[3] == 'u') return 3;
    return e[0] == '2' ? 2 : 1;
  }();
  return sel;
}
template <int VPL, int U>
// With `dependent`, the gather is launched as a programmatic dependent of the
// kernel before it on `st` (the plan): its launch and CTA placement overlap the
// plan's tail, and it waits for the plan grid before reading its tables.
static sns_status launch_warp_gather_t(const DenseArgs& a, int64_t d, const CsLayout& L, uint8_t* ws, float* SA,
                                       int64_t ldsa, float* Sb, int64_t sbs, cudaStream_t st, bool dependent) {
  constexpr int CT = 128 * VPL;
  const int64_t ntile = (a.n + CT - 1) / CT;
  auto kern = cs_gather_warp<VPL, U>;
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0));
  const int64_t grid2 = (int64_t)num_sms() * std::max(occ, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid2);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = dependent ? 1 : 0;
  {
    SNS_PROF(K_CS_GATHER, st);
    SNS_CUDA_TRY(cudaLaunchKernelEx(
        &cfg, kern, static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b), a.n, ntile,
        reinterpret_cast<const uint32_t*>(ws + L.off_list), reinterpret_cast<const uint32_t*>(ws + L.off_btot),
        reinterpret_cast<const uint32_t*>(ws + L.off_bbase), reinterpret_cast<const uint32_t*>(ws + L.off_cbase),
        reinterpret_cast<const uint32_t*>(ws + L.off_ctab), (uint32_t)d, reinterpret_cast<uint32_t*>(ws + L.off_ticket),
        reinterpret_cast<uint32_t*>(ws + L.off_err) + 1, reinterpret_cast<float*>(ws + L.off_wpart), SA, ldsa, Sb,
        sbs, reinterpret_cast<const int*>(ws + L.off_err)));
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}
static sns_status launch_warp_gather(const DenseArgs& a, int64_t d, const CsLayout& L, uint8_t* ws, float* SA,
                                     int64_t ldsa, float* Sb, int64_t sbs, cudaStream_t st, bool dependent = false) {
  int choice = warp_tile_choice();
  if (choice == 0) choice = a.n > 128 ? 2 : 1;
  switch (choice) {
    case 2: return launch_warp_gather_t<2, 8>(a, d, L, ws, SA, ldsa, Sb, sbs, st, dependent);
    case 3: return launch_warp_gather_t<2, 4>(a, d, L, ws, SA, ldsa, Sb, sbs, st, dependent);
    default: return launch_warp_gather_t<1, 8>(a, d, L, ws, SA, ldsa, Sb, sbs, st, dependent);
  }
}

sns_status cs_tma_phase2(const DenseArgs& a, int64_t d, const CsLayout& L, uint8_t* ws, float* SA, int64_t ldsa,
                         float* Sb, int64_t sbs, cudaStream_t st, bool allow_bulk) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((d + 7) / 8, (int64_t)num_sms() * 4));
  const size_t smem = (size_t)d * 8;
  SNS_CUDA_TRY(raise_smem_limit((const void*)cs_build_list));
  uint32_t* cbase = reinterpret_cast<uint32_t*>(ws + L.off_cbase);
  uint32_t* ctab = reinterpret_cast<uint32_t*>(ws + L.off_ctab);
  const bool use_tma = allow_bulk && cs_bulk_gather_selected();
  {
    SNS_PROF(K_CS_SORT, st);
    cs_build_list<<<grid, 256, smem, st>>>((uint32_t)d, L.nblk, reinterpret_cast<const uint32_t*>(ws + L.off_sorted),
                                           reinterpret_cast<const uint32_t*>(ws + L.off_seg),
                                           reinterpret_cast<const uint32_t*>(ws + L.off_btot),
                                           reinterpret_cast<uint32_t*>(ws + L.off_bbase),
                                           reinterpret_cast<uint32_t*>(ws + L.off_list), cbase, ctab,
                                           use_tma ? nullptr : SA, ldsa, Sb, sbs, a.n);
  }
  SNS_LAUNCH_CHECK();
  if (use_tma)
    return a.n <= 128 ? launch_tma<128>(a, d, L, ws, SA, ldsa, Sb, sbs, st)
                      : launch_tma<256>(a, d, L, ws, SA, ldsa, Sb, sbs, st);
  return launch_warp_gather(a, d, L, ws, SA, ldsa, Sb, sbs, st);
}

bool cs_bulk_gather_selected() {
  static const bool sel = [] {
    const char* e = getenv("SNSOLVE_CS_GATHER");
    return e && e[0] == 't';
  }();
  return sel;
}

// Plan (cs_plan_coop, cooperative) + warp gather.  *used = false (nothing
// launched) when the blocks cannot all be co-resident; the caller then runs
// the two-kernel plan.  Error word layout (16 bytes at L.off_err): [0] error,
// [1] gather item counter, [2] grid-barrier arrivals.
sns_status cs_coop_apply(const DenseArgs& a, int64_t d, uint64_t seed, const CsLayout& L, uint8_t* ws, float* SA,
                         int64_t ldsa, float* Sb, int64_t sbs, cudaStream_t st, bool* used) {
  *used = false;
  // ranks and offsets within a block are 16-bit; a block of at least 4096
  // rows keeps the block totals within the two-kernel plan's table
  const int64_t rows_per_blk = kListRowsPerBlock;
  const int64_t nblk_plan = (a.m + rows_per_blk - 1) / rows_per_blk;
  const size_t smem = cs_plan_smem(d, rows_per_blk);
  SNS_CUDA_TRY(raise_smem_limit((const void*)cs_plan_coop));
  int dev = 0, smem_max = 0;
  SNS_CUDA_TRY(cudaGetDevice(&dev));
  SNS_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 1024 > (size_t)smem_max) return SNS_OK;
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cs_plan_coop, kPlanWarps * 32, smem));
  if ((int64_t)occ * num_sms() < nblk_plan || nblk_plan > L.nblk) return SNS_OK;
  *used = true;
  SNS_CUDA_TRY(cudaMemsetAsync(ws + L.off_err, 0, 16, st));
  ProfSpan span(K_CS_APPLY, st);                   // plan + gather, timed as one
  int64_t m = a.m, nblk = nblk_plan, nticket = L.nticket, n = a.n, ldsa_ = ldsa, sbs_ = sbs;
  int rpb = (int)rows_per_blk;
  uint32_t dd = (uint32_t)d;
  uint64_t s0 = shift_state(stream_state(seed, kStreamCountSketch), a.row0);
  uint32_t* seg = reinterpret_cast<uint32_t*>(ws + L.off_seg);
  uint32_t* ticket = reinterpret_cast<uint32_t*>(ws + L.off_ticket);
  uint32_t* btot = reinterpret_cast<uint32_t*>(ws + L.off_btot);
  uint32_t* bbase = reinterpret_cast<uint32_t*>(ws + L.off_bbase);
  uint32_t* list = reinterpret_cast<uint32_t*>(ws + L.off_list);
  uint32_t* cbase = reinterpret_cast<uint32_t*>(ws + L.off_cbase);
  uint32_t* ctab = reinterpret_cast<uint32_t*>(ws + L.off_ctab);
  uint32_t* bar = reinterpret_cast<uint32_t*>(ws + L.off_err) + 2;
  int* err = reinterpret_cast<int*>(ws + L.off_err);
  int nbits = 1;                                   // bit length of d
  while (((int64_t)1 << nbits) <= d) ++nbits;
  void* args[] = {&m, &dd, &s0, &nblk, &seg, &ticket, &nticket, &btot, &bbase, &list, &cbase, &ctab,
                  &SA, &ldsa_, &Sb, &sbs_, &n, &bar, &err, &nbits, &rpb};
  {
    SNS_PROF(K_CS_SORT, st);
    SNS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)cs_plan_coop, dim3((unsigned)nblk), dim3(kPlanWarps * 32),
                                             args, smem, st));
  }
  return launch_warp_gather(a, d, L, ws, SA, ldsa, Sb, sbs, st, /*dependent=*/true);
}

}  // namespace sns
