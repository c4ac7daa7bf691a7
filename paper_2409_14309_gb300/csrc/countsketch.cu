// CountSketch apply (Clarkson-Woodruff sketch, Sec. 1.2.2 of arXiv 2409.14309;
// the paper's default operator): SA[h(i), :] += s(i) * A[i, :], Sb[h(i)] += s(i) * b[i].
//
// Two dense variants and one CSR variant:
//  * sorted (deterministic): phase 1 hashes every row and counting-sorts the
//    row ids of each block of kRowsPerBlock rows by bucket (stable, so rows of
//    a bucket stay in ascending order); phase 2 gives each CTA a slice of one
//    bucket's rows, sums them in registers (rows are whole 1 KB-class
//    contiguous reads), and the last CTA of a bucket adds the slices in a
//    fixed order.  Bitwise reproducible for a fixed (m, d, n).
//  * stream: one pass over A in row order; each warp adds its signed rows into
//    SA with vector reductions (red.global.add.v4.f32) that land in L2.
//  * CSR: phase 1 as above; phase 2 accumulates the sparse rows of a bucket
//    slice into per-warp shared-memory rows (equal columns of one step added
//    in lane order), then combines as above: bitwise reproducible too.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "prof.h"

namespace sns {

constexpr int kRowsPerBlock = 4096;      // rows per phase-1 block (segment source)
constexpr int kSortWarps = 8;
constexpr int kGatherWarps = 8;
constexpr int kGatherU = 4;              // rows in flight per warp
constexpr int kRowsPerItem = 256;        // target rows per phase-2 work item
constexpr uint16_t kNoBucket = 0xFFFF;

int64_t cs_nblk(int64_t m) { return (m + kRowsPerBlock - 1) / kRowsPerBlock; }

// Segments (phase-1 blocks) per phase-2 item so an item holds ~kRowsPerItem rows.
static int64_t cs_seg_per_item(int64_t m, int64_t d) {
  const int64_t nblk = cs_nblk(m);
  double rows_per_seg = (double)m / (double)(nblk * d);
  int64_t spi = (int64_t)((double)kRowsPerItem / (rows_per_seg > 0 ? rows_per_seg : 1.0)) + 1;
  if (spi > nblk) spi = nblk;
  if (spi < 1) spi = 1;
  return spi;
}

CsLayout cs_layout(int64_t m, int64_t n, int64_t d, bool f64, bool csr) {
  CsLayout L{};
  L.nblk = cs_nblk(m);
  L.spi = cs_seg_per_item(m, d);
  L.parts = (L.nblk + L.spi - 1) / L.spi;
  const int64_t ct = csr ? n : (f64 ? 128 : (n <= 128 ? 128 : 256));
  L.ct = ct;
  L.ntile = csr ? 1 : (n + ct - 1) / ct;
  const int64_t esz = f64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  L.off_sorted = take((size_t)L.nblk * kRowsPerBlock * 4);
  L.off_seg = take((size_t)L.nblk * d * 4);
  L.nticket = d * std::max<int64_t>(L.ntile, (n + 127) / 128);   // >= d * ceil(n / 128) for every phase 2
  L.off_ticket = take((size_t)L.nticket * 4);
  // partial rows: one per (bucket, part, tile), each ct values + 1 for b; sized
  // for both phase-2 kernels (the bulk-copy one uses its own part count)
  L.tma_parts = (csr || f64) ? 1 : cs_tma_parts(m, d);
  const int64_t tma_ct = n <= 128 ? 128 : 256, tma_ntile = (n + tma_ct - 1) / tma_ct;
  const size_t part_a = L.parts > 1 ? (size_t)d * L.parts * L.ntile * (ct + 1) * esz : 0;
  const size_t part_b = L.tma_parts > 1 ? (size_t)d * L.tma_parts * tma_ntile * (tma_ct + 1) * 4 : 0;
  L.off_part = take(std::max(part_a, part_b));
  L.off_list = take((csr || f64) ? 0 : (size_t)m * 4);
  L.off_btot = take((size_t)d * 4);
  L.off_bbase = take((size_t)d * 4);
  L.off_err = take(16);
  // warp-gather chunk tables and chunk partial rows (dense FP32 only)
  const bool wg = !(csr || f64);
  const int64_t maxch = wg ? cs_warp_max_chunks(m, d) : 0;
  L.off_cbase = take(wg ? (size_t)(d + 1) * 4 : 0);
  L.off_ctab = take((size_t)maxch * 4);
  // chunk partial rows of the warp gather, for either column tile (128 or 256)
  L.off_wpart = take((size_t)maxch * std::max<int64_t>(((n + 127) / 128) * (128 + 4), ((n + 255) / 256) * (256 + 4)) * 4);
  L.bytes = off;
  return L;
}

// ---------------------------------------------------------------------------
// Phase 1: per block of kRowsPerBlock rows, hash, per-warp histograms (no
// atomics: match_any groups equal buckets), bucket offsets, stable scatter.
// Writes sorted[blk*R + pos] = row | (sign bit << 31) and
// seg[k * nblk + blk] = (start << 16) | count.  Also clears the tickets.
__global__ void __launch_bounds__(kSortWarps * 32)
cs_sort_blocks(int64_t m, uint32_t d, uint64_t s0, int64_t nblk, uint32_t* __restrict__ sorted,
               uint32_t* __restrict__ seg, uint32_t* __restrict__ ticket, int64_t nticket, uint32_t* __restrict__ btot) {
  extern __shared__ __align__(16) uint8_t smraw[];
  uint16_t* cnt = reinterpret_cast<uint16_t*>(smraw);              // [W][d]
  uint16_t* hb = cnt + (size_t)kSortWarps * d;                      // [R]
  __shared__ uint32_t wsum[kSortWarps * 32 / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t blk = blockIdx.x;
  const int64_t r0 = blk * kRowsPerBlock;
  constexpr int kRowsPerWarp = kRowsPerBlock / kSortWarps;

  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + tid; i < nticket; i += (int64_t)gridDim.x * blockDim.x)
    ticket[i] = 0;
  for (int i = tid; i < kSortWarps * (int)d; i += blockDim.x) cnt[i] = 0;
  __syncthreads();

  // hb keeps the bucket (bits 0..14; d <= 8192) and the sign (bit 15), so the
  // scatter below does not hash again
  for (int j = 0; j < kRowsPerWarp; j += 32) {
    const int loc = w * kRowsPerWarp + j + lane;
    const int64_t row = r0 + loc;
    uint32_t h = kNoBucket;
    uint32_t sgn = 0;
    if (row < m) {
      const uint64_t key = splitmix_at(s0, (uint64_t)row);
      h = bucket_of(key, d);
      sgn = (uint32_t)(key >> 63);
    }
    hb[loc] = (uint16_t)(h == kNoBucket ? kNoBucket : (h | (sgn << 15)));
    const unsigned peers = __match_any_sync(0xffffffffu, h);
    if (h != kNoBucket && lane == __ffs(peers) - 1) cnt[w * d + h] += (uint16_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // Per-bucket totals and exclusive scan over buckets (each thread owns a
  // contiguous run of buckets), then per-warp starting offsets in place.
  const int nt = blockDim.x;
  const int per = ((int)d + nt - 1) / nt;
  const int k0 = tid * per;
  const int k1 = min((int)d, k0 + per);
  uint32_t local = 0;
  for (int k = k0; k < k1; ++k)
    for (int ww = 0; ww < kSortWarps; ++ww) local += cnt[ww * d + k];
  // block exclusive scan of `local`
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  uint32_t base = 0;
  for (int ww = 0; ww < w; ++ww) base += wsum[ww];
  uint32_t running = base + incl - local;
  for (int k = k0; k < k1; ++k) {
    uint32_t tot = 0;
    for (int ww = 0; ww < kSortWarps; ++ww) {
      const uint32_t c = cnt[ww * d + k];
      cnt[ww * d + k] = (uint16_t)(running + tot);
      tot += c;
    }
    seg[(size_t)k * nblk + blk] = (running << 16) | tot;
    if (tot) atomicAdd(btot + k, tot);   // bucket totals (integer adds: order does not matter)
    running += tot;
  }
  __syncthreads();

  // Stable scatter: a warp walks its rows in order; equal buckets inside a
  // 32-row chunk are ranked by lane.
  const unsigned lt = (1u << lane) - 1u;
  for (int j = 0; j < kRowsPerWarp; j += 32) {
    const int loc = w * kRowsPerWarp + j + lane;
    const int64_t row = r0 + loc;
    const uint32_t hw = hb[loc];
    const uint32_t h = hw == kNoBucket ? kNoBucket : (hw & 0x7FFFu);
    const unsigned peers = __match_any_sync(0xffffffffu, h);
    uint32_t pos = 0;
    if (h != kNoBucket) {
      pos = cnt[w * d + h] + __popc(peers & lt);
      sorted[r0 + pos] = (uint32_t)row | ((hw >> 15) << 31);
    }
    __syncwarp();
    if (h != kNoBucket && lane == __ffs(peers) - 1) cnt[w * d + h] += (uint16_t)__popc(peers);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Expand the segments of one warp into row ids, 32 at a time.
// Segment t of the warp (t = 0..31) is block blk_l of lane t; its rows are
// sorted[blk_l*R + st_l .. + cnt_l).  Lane l receives row number j0 + l of the
// concatenation, or 0xFFFFFFFF past the end.
struct SegSet {
  uint32_t incl, st;
  int64_t blk;
  uint32_t total;
};
SNS_D SegSet load_segs(const uint32_t* __restrict__ seg, int64_t k, int64_t nblk, int64_t blk_l, bool valid) {
  const int lane = threadIdx.x & 31;
  uint32_t sv = valid ? __ldg(seg + (size_t)k * nblk + blk_l) : 0u;
  uint32_t c = sv & 0xFFFFu;
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  SegSet S;
  S.incl = incl;
  S.st = sv >> 16;
  S.blk = blk_l;
  S.total = __shfl_sync(0xffffffffu, incl, 31);
  return S;
}
SNS_D uint32_t seg_row(const SegSet& S, const uint32_t* __restrict__ sorted, uint32_t j) {
  // q = number of lanes whose inclusive prefix is <= j
  int q = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const uint32_t v = __shfl_sync(0xffffffffu, S.incl, q + s - 1);
    if (v <= j) q += s;
  }
  // every lane executes every shuffle (full-mask shuffles must not diverge)
  const uint32_t st_q = __shfl_sync(0xffffffffu, S.st, q);
  const int64_t blk_q = __shfl_sync(0xffffffffu, S.blk, q);
  const uint32_t prev = __shfl_sync(0xffffffffu, S.incl, q > 0 ? q - 1 : 0);
  const uint32_t excl_q = (q > 0) ? prev : 0u;
  if (j >= S.total) return 0xFFFFFFFFu;
  return __ldg(sorted + blk_q * kRowsPerBlock + st_q + (j - excl_q));
}
// NOTE: seg_row must be called by all 32 lanes (it shuffles); lanes past the
// end get 0xFFFFFFFF.

template <typename T, int VEC>
struct VecT;
template <>
struct VecT<float, 4> {
  using type = float4;
};
template <>
struct VecT<float, 1> {
  using type = float;
};
template <>
struct VecT<double, 2> {
  using type = double2;
};
template <>
struct VecT<double, 1> {
  using type = double;
};

template <typename T, int VEC>
SNS_D void load_vec(const T* p, T (&v)[VEC]) {
  if constexpr (VEC == 4) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (VEC == 2) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = __ldg(p);
  }
}

// Phase 2 (dense): work item = (bucket k, part p, column tile t).  Warps take
// the item's segments round-robin, accumulate kGatherU independent partial
// rows each (rows in ascending order inside a segment), then the CTA adds all
// partials in a fixed tree order.  If the bucket has several parts, the part
// row goes to workspace and the last CTA to finish the bucket (ticket) adds the
// parts in part order.
template <typename T, int VEC, int NCH>
__global__ void __launch_bounds__(kGatherWarps * 32)
cs_gather_dense(const T* __restrict__ A, int64_t lda, const T* __restrict__ b, int64_t n, uint32_t d,
                int64_t nblk, int64_t spi, int64_t parts, int64_t ntile,
                const uint32_t* __restrict__ sorted, const uint32_t* __restrict__ seg,
                uint32_t* __restrict__ ticket, T* __restrict__ part_buf,
                T* __restrict__ SA, int64_t ldsa, T* __restrict__ Sb, int64_t sbs) {
  constexpr int CT = 32 * VEC * NCH;
  constexpr int NP = kGatherWarps * kGatherU;          // partial rows per CTA
  extern __shared__ __align__(16) uint8_t smraw[];
  T* red = reinterpret_cast<T*>(smraw);                // [NP][CT + 1]
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nitems = (int64_t)d * parts * ntile;

  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int64_t t = item % ntile;
    const int64_t kp = item / ntile;
    const int64_t p = kp % parts;
    const int64_t k = kp / parts;
    const int64_t col0 = t * CT;
    const int64_t sb0 = p * spi, sb1 = min(nblk, sb0 + spi);

    T acc[kGatherU][NCH][VEC];
    T accb[kGatherU];
#pragma unroll
    for (int u = 0; u < kGatherU; ++u) {
      accb[u] = T(0);
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[u][q][v] = T(0);
    }
    bool colok[NCH];
#pragma unroll
    for (int q = 0; q < NCH; ++q) colok[q] = (col0 + q * 32 * VEC + lane * VEC) < n;

    for (int64_t sbase = sb0 + w; sbase < sb1; sbase += (int64_t)kGatherWarps * 32) {
      const int64_t blk_l = sbase + (int64_t)lane * kGatherWarps;
      const SegSet S = load_segs(seg, k, nblk, blk_l, blk_l < sb1);
      for (uint32_t j0 = 0; j0 < S.total; j0 += 32) {
        const uint32_t rid_l = seg_row(S, sorted, j0 + lane);
        const int nr = (int)min(32u, S.total - j0);
        for (int r = 0; r < nr; r += kGatherU) {
          T x[kGatherU][NCH][VEC];
          T xb[kGatherU];
          uint32_t rid[kGatherU];
#pragma unroll
          for (int u = 0; u < kGatherU; ++u) {
            rid[u] = __shfl_sync(0xffffffffu, rid_l, (r + u) & 31);
            const bool ok = (r + u) < nr;
            const int64_t row = (int64_t)(rid[u] & 0x7FFFFFFFu);
            const T* rp = A + row * lda + col0 + lane * VEC;
#pragma unroll
            for (int q = 0; q < NCH; ++q) {
              if (ok && colok[q]) {
                load_vec<T, VEC>(rp + q * 32 * VEC, x[u][q]);
              } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) x[u][q][v] = T(0);
              }
            }
            xb[u] = (ok && t == 0 && lane == 0) ? __ldg(b + row) : T(0);
          }
#pragma unroll
          for (int u = 0; u < kGatherU; ++u) {
            const bool neg = (rid[u] >> 31) != 0;
#pragma unroll
            for (int q = 0; q < NCH; ++q)
#pragma unroll
              for (int v = 0; v < VEC; ++v) acc[u][q][v] += neg ? -x[u][q][v] : x[u][q][v];
            accb[u] += neg ? -xb[u] : xb[u];
          }
        }
      }
    }
    // partial rows -> shared memory
#pragma unroll
    for (int u = 0; u < kGatherU; ++u) {
      T* rr = red + (size_t)(w * kGatherU + u) * (CT + 1);
#pragma unroll
      for (int q = 0; q < NCH; ++q)
#pragma unroll
        for (int v = 0; v < VEC; ++v) rr[q * 32 * VEC + lane * VEC + v] = acc[u][q][v];
      if (lane == 0) rr[CT] = accb[u];
    }
    __syncthreads();
    // fixed-order pairwise tree over the NP partial rows
    for (int c = threadIdx.x; c <= CT; c += blockDim.x) {
      T vals[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) vals[i] = red[(size_t)i * (CT + 1) + c];
#pragma unroll
      for (int s = NP / 2; s > 0; s >>= 1)
#pragma unroll
        for (int i = 0; i < s; ++i) vals[i] += vals[i + s];
      red[c] = vals[0];
    }
    __syncthreads();
    if (parts == 1) {
      for (int c = threadIdx.x; c < CT; c += blockDim.x)
        if (col0 + c < n) SA[k * ldsa + col0 + c] = red[c];
      if (t == 0 && threadIdx.x == 0) Sb[k * sbs] = red[CT];
    } else {
      T* pb = part_buf + ((size_t)(k * ntile + t) * parts + p) * (CT + 1);
      for (int c = threadIdx.x; c <= CT; c += blockDim.x) pb[c] = red[c];
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(ticket + k * ntile + t, 1u) == (uint32_t)(parts - 1));
      __syncthreads();
      if (s_last) {
        __threadfence();
        const T* pk = part_buf + (size_t)(k * ntile + t) * parts * (CT + 1);
        for (int c = threadIdx.x; c <= CT; c += blockDim.x) {
          T s = T(0);
          for (int64_t pp = 0; pp < parts; ++pp) s += __ldcg(pk + pp * (CT + 1) + c);
          if (c < CT) {
            if (col0 + c < n) SA[k * ldsa + col0 + c] = s;
          } else if (t == 0) {
            Sb[k * sbs] = s;
          }
        }
      }
    }
    __syncthreads();
  }
}

// Phase 2 (CSR): a lane takes a whole sparse row and adds it into its warp's
// shared row accumulator (n floats + 1 for b); lanes that hit the same column
// in one step add in lane order, the warps' rows are added in warp order and
// the parts in part order, so the result is bitwise reproducible.
__global__ void __launch_bounds__(kGatherWarps * 32)
cs_gather_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
              const float* __restrict__ b, int64_t n, uint32_t d, int64_t nblk, int64_t spi, int64_t parts,
              const uint32_t* __restrict__ sorted, const uint32_t* __restrict__ seg,
              uint32_t* __restrict__ ticket, float* __restrict__ part_buf,
              float* __restrict__ SA, int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  extern __shared__ __align__(16) uint8_t smraw[];
  float* accs = reinterpret_cast<float*>(smraw);   // [kGatherWarps][n + 1]: one row per warp
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  float* acc = accs + (size_t)w * (n + 1);
  const int64_t nitems = (int64_t)d * parts;
  for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int64_t p = item % parts, k = item / parts;
    const int64_t sb0 = p * spi, sb1 = min(nblk, sb0 + spi);
    for (int64_t c = threadIdx.x; c < (int64_t)kGatherWarps * (n + 1); c += blockDim.x) accs[c] = 0.f;
    __syncthreads();
    for (int64_t sbase = sb0 + w; sbase < sb1; sbase += (int64_t)kGatherWarps * 32) {
      const int64_t blk_l = sbase + (int64_t)lane * kGatherWarps;
      const SegSet S = load_segs(seg, k, nblk, blk_l, blk_l < sb1);
      for (uint32_t j0 = 0; j0 < S.total; j0 += 32) {
        const uint32_t rid = seg_row(S, sorted, j0 + lane);
        const bool okr = rid != 0xFFFFFFFFu;
        const int64_t row = okr ? (int64_t)(rid & 0x7FFFFFFFu) : 0;
        const float sg = (rid >> 31) ? -1.f : 1.f;
        int64_t e = okr ? __ldg(rowptr + row) : 0;
        const int64_t e1 = okr ? __ldg(rowptr + row + 1) : 0;
        const float bv = okr ? sg * __ldg(b + row) : 0.f;
        // the lanes' rows 8 entries at a time, warp-uniform; lanes that hit the
        // same column add in lane order (one shared store per round), so every
        // address sees its additions in a fixed order
        while (__any_sync(0xffffffffu, e < e1)) {
          int32_t cc[8];
          float vv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const bool ok = e + u < e1;
            cc[u] = ok ? __ldg(col + e + u) : -1;
            vv[u] = ok ? __ldg(val + e + u) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const unsigned peers = __match_any_sync(0xffffffffu, cc[u]);
            const int rank = cc[u] >= 0 ? __popc(peers & lt) : 0;
            const int rounds = __reduce_max_sync(0xffffffffu, (unsigned)rank) + 1;
            for (int rr = 0; rr < rounds; ++rr) {
              if (cc[u] >= 0 && rank == rr) acc[cc[u]] += sg * vv[u];
              __syncwarp();
            }
          }
          e += 8;
        }
        const float bs = warp_sum(bv);                    // fixed reduction tree
        if (lane == 0) acc[n] += bs;
        __syncwarp();
      }
    }
    __syncthreads();
    // the warps' rows in warp order
    auto total = [&](int64_t c) {
      float t = 0.f;
#pragma unroll
      for (int ww = 0; ww < kGatherWarps; ++ww) t += accs[(size_t)ww * (n + 1) + c];
      return t;
    };
    if (parts == 1) {
      for (int64_t c = threadIdx.x; c < n; c += blockDim.x) SA[k * ldsa + c] = total(c);
      if (threadIdx.x == 0) Sb[k * sbs] = total(n);
    } else {
      float* pb = part_buf + ((size_t)k * parts + p) * (n + 1);
      for (int64_t c = threadIdx.x; c <= n; c += blockDim.x) pb[c] = total(c);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = (atomicAdd(ticket + k, 1u) == (uint32_t)(parts - 1));
      __syncthreads();
      if (s_last) {
        __threadfence();
        const float* pk = part_buf + (size_t)k * parts * (n + 1);
        for (int64_t c = threadIdx.x; c <= n; c += blockDim.x) {
          float s = 0.f;
          for (int64_t pp = 0; pp < parts; ++pp) s += __ldcg(pk + pp * (n + 1) + c);
          if (c < n) SA[k * ldsa + c] = s; else Sb[k * sbs] = s;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Streaming variant (FP32 only): rows in order, each warp adds kGatherU signed
// rows at a time into SA with vector reductions.  SA and Sb must be zeroed.
template <int VEC>
__global__ void __launch_bounds__(256)
cs_stream_dense(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n,
                uint32_t d, uint64_t s0, float* __restrict__ SA, int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = gw * kGatherU; r0 < m; r0 += nw * kGatherU) {
    uint32_t h[kGatherU];
    bool neg[kGatherU];
#pragma unroll
    for (int u = 0; u < kGatherU; ++u) {
      const int64_t row = r0 + u;
      const uint64_t key = splitmix_at(s0, (uint64_t)(row < m ? row : 0));
      h[u] = bucket_of(key, d);
      neg[u] = (key >> 63) != 0;
    }
    for (int64_t c0 = (int64_t)lane * VEC; c0 < n; c0 += 32 * VEC) {
      float x[kGatherU][VEC];
#pragma unroll
      for (int u = 0; u < kGatherU; ++u) {
        if (r0 + u < m) {
          load_vec<float, VEC>(A + (r0 + u) * lda + c0, x[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kGatherU; ++u) {
        if (r0 + u >= m) continue;
        float* dst = SA + (int64_t)h[u] * ldsa + c0;
        const float sg = neg[u] ? -1.f : 1.f;
        if constexpr (VEC == 4) {
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(sg * x[u][0]),
                       "f"(sg * x[u][1]), "f"(sg * x[u][2]), "f"(sg * x[u][3])
                       : "memory");
        } else {
          atomicAdd(dst, sg * x[u][0]);
        }
      }
    }
    if (lane < kGatherU && r0 + lane < m) {
      float hb = 0.f;
      uint32_t hh = 0;
      bool ng = false;
#pragma unroll
      for (int u = 0; u < kGatherU; ++u)
        if (u == lane) { hh = h[u]; ng = neg[u]; }
      hb = __ldg(b + r0 + lane);
      atomicAdd(Sb + (int64_t)hh * sbs, ng ? -hb : hb);
    }
  }
}

// ---------------------------------------------------------------------------
// Sparse sign embedding (Sec. 1.2.2, after Martinsson & Tropp 2020), dense
// FP32: column i of S holds zeta nonzeros +-1/sqrt(zeta) at distinct rows.
// Draw z of row i uses output i of stream 0 (z = 0, so zeta = 1 is the
// CountSketch) or output i*(zeta-1) + z-1 of stream 4; the rows follow Floyd's
// algorithm on [0, d) (draw z takes u = ((k mod 2^32) * (J + 1)) >> 32,
// J = d - zeta + z, or J if an earlier draw of the row took u) and the sign of
// draw z is bit 63 of its key.  One streaming pass: each warp takes kSseRows
// rows at a time and adds every row into its zeta rows of SA with vector
// reductions.  SA and Sb must be zeroed.
constexpr int kSseMaxZeta = 8;
constexpr int kSseRows = 2;
template <int VEC>
__global__ void __launch_bounds__(256)
cs_sparse_sign_dense(const float* __restrict__ A, int64_t lda, const float* __restrict__ b, int64_t m, int64_t n,
                     uint32_t d, int zeta, uint64_t s0, uint64_t s4, float scale, float* __restrict__ SA,
                     int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = gw * kSseRows; r0 < m; r0 += nw * kSseRows) {
    uint32_t h[kSseRows][kSseMaxZeta];
    float sg[kSseRows][kSseMaxZeta];
#pragma unroll
    for (int u = 0; u < kSseRows; ++u) {
      const uint64_t row = (uint64_t)(r0 + u < m ? r0 + u : 0);
#pragma unroll
      for (int z = 0; z < kSseMaxZeta; ++z) {
        h[u][z] = 0u;
        sg[u][z] = 0.f;
        if (z < zeta) {
          const uint64_t key = z == 0 ? splitmix_at(s0, row) : splitmix_at(s4, row * (uint64_t)(zeta - 1) + (z - 1));
          const uint32_t J = d - (uint32_t)zeta + (uint32_t)z;
          const uint32_t cand = (uint32_t)(((key & 0xFFFFFFFFull) * ((uint64_t)J + 1)) >> 32);
          bool taken = false;
#pragma unroll
          for (int zz = 0; zz < z; ++zz) taken = taken || (h[u][zz] == cand);
          h[u][z] = taken ? J : cand;
          sg[u][z] = (key >> 63) ? -scale : scale;
        }
      }
    }
    for (int64_t c0 = (int64_t)lane * VEC; c0 < n; c0 += 32 * VEC) {
      float x[kSseRows][VEC];
#pragma unroll
      for (int u = 0; u < kSseRows; ++u)
        if (r0 + u < m) load_vec<float, VEC>(A + (r0 + u) * lda + c0, x[u]);
#pragma unroll
      for (int u = 0; u < kSseRows; ++u) {
        if (r0 + u >= m) continue;
#pragma unroll
        for (int z = 0; z < kSseMaxZeta; ++z) {
          if (z >= zeta) break;
          float* dst = SA + (int64_t)h[u][z] * ldsa + c0;
          const float f = sg[u][z];
          if constexpr (VEC == 4) {
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(f * x[u][0]),
                         "f"(f * x[u][1]), "f"(f * x[u][2]), "f"(f * x[u][3])
                         : "memory");
          } else {
            atomicAdd(dst, f * x[u][0]);
          }
        }
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < kSseRows; ++u) {
        if (r0 + u >= m) continue;
        const float bv = __ldg(b + r0 + u);
#pragma unroll
        for (int z = 0; z < kSseMaxZeta; ++z)
          if (z < zeta) atomicAdd(Sb + (int64_t)h[u][z] * sbs, sg[u][z] * bv);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// SM count of the current device, cached per device index (grids are sized
// from it, so a process that drives several devices needs each one's own).
constexpr int kMaxSmDevices = 64;
static std::atomic<int> g_num_sms[kMaxSmDevices];
int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  std::atomic<int>* slot = dev < kMaxSmDevices ? &g_num_sms[dev] : nullptr;
  int v = slot ? slot->load(std::memory_order_relaxed) : 0;
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
  if (slot) slot->store(v, std::memory_order_relaxed);   // every racing writer stores the same value
  return v;
}

static size_t sort_smem(int64_t d) { return (size_t)kSortWarps * d * 2 + (size_t)kRowsPerBlock * 2; }

sns_status cs_phase1(int64_t m, int64_t d, uint64_t seed, int64_t row0, const CsLayout& L, uint8_t* ws,
                     cudaStream_t st) {
  const size_t smem = sort_smem(d);
  SNS_CUDA_TRY(cudaMemsetAsync(ws + L.off_btot, 0, (size_t)d * 4, st));
  SNS_CUDA_TRY(cudaMemsetAsync(ws + L.off_err, 0, 16, st));   // error word and phase-2 item counter
  SNS_CUDA_TRY(raise_smem_limit((const void*)cs_sort_blocks));
  {
    SNS_PROF(K_CS_SORT, st);
  cs_sort_blocks<<<(unsigned)L.nblk, kSortWarps * 32, smem, st>>>(
      m, (uint32_t)d, shift_state(stream_state(seed, kStreamCountSketch), row0), L.nblk,
      reinterpret_cast<uint32_t*>(ws + L.off_sorted),
      reinterpret_cast<uint32_t*>(ws + L.off_seg), reinterpret_cast<uint32_t*>(ws + L.off_ticket),
      L.nticket, reinterpret_cast<uint32_t*>(ws + L.off_btot));
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

template <typename T, int VEC, int NCH>
static sns_status launch_gather(const DenseArgs& a, int64_t d, const CsLayout& L, uint8_t* ws, void* SA, int64_t ldsa,
                                void* Sb, int64_t sbs, cudaStream_t st) {
  constexpr int CT = 32 * VEC * NCH;
  const size_t smem = (size_t)kGatherWarps * kGatherU * (CT + 1) * sizeof(T);
  auto kern = cs_gather_dense<T, VEC, NCH>;
  SNS_CUDA_TRY(raise_smem_limit((const void*)kern));
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGatherWarps * 32, smem));
  if (occ < 1) occ = 1;
  const int64_t items = d * L.parts * L.ntile;
  const int64_t grid = std::min<int64_t>(items, (int64_t)num_sms() * occ);
  {
    SNS_PROF(K_CS_GATHER, st);
  kern<<<(unsigned)grid, kGatherWarps * 32, smem, st>>>(
      static_cast<const T*>(a.A), a.lda, static_cast<const T*>(a.b), a.n, (uint32_t)d, L.nblk, L.spi, L.parts,
      L.ntile, reinterpret_cast<const uint32_t*>(ws + L.off_sorted), reinterpret_cast<const uint32_t*>(ws + L.off_seg),
      reinterpret_cast<uint32_t*>(ws + L.off_ticket), reinterpret_cast<T*>(ws + L.off_part), static_cast<T*>(SA), ldsa,
      static_cast<T*>(Sb), sbs);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

sns_status cs_apply_dense_sorted(const DenseArgs& a, int64_t d, uint64_t seed, void* SA, int64_t ldsa, void* Sb,
                                 int64_t sbs, void* ws, size_t ws_bytes, cudaStream_t st, bool allow_bulk) {
  const CsLayout L = cs_layout(a.m, a.n, d, a.f64, false);
  if (ws_bytes < L.bytes) return SNS_ENOMEM;
  uint8_t* w = static_cast<uint8_t*>(ws);
  sns_status s;
  if (!a.f64 && allow_bulk && cs_tma_eligible(a) && !cs_bulk_gather_selected()) {
    // one cooperative plan launch (bounded grid barriers) + the warp gather
    bool used = false;
    s = cs_coop_apply(a, d, seed, L, w, static_cast<float*>(SA), ldsa, static_cast<float*>(Sb), sbs, st, &used);
    if (s != SNS_OK || used) return s;
  }
  s = cs_phase1(a.m, d, seed, a.row0, L, w, st);
  if (s != SNS_OK) return s;
  if (a.f64) {
    const bool v2 = (a.lda % 2 == 0) && aligned(a.A, 16);
    return v2 ? launch_gather<double, 2, 2>(a, d, L, w, SA, ldsa, Sb, sbs, st)
              : launch_gather<double, 1, 4>(a, d, L, w, SA, ldsa, Sb, sbs, st);
  }
  if (cs_tma_eligible(a))
    return cs_tma_phase2(a, d, L, w, static_cast<float*>(SA), ldsa, static_cast<float*>(Sb), sbs, st, allow_bulk);
  const bool v4 = (a.lda % 4 == 0) && aligned(a.A, 16);
  if (L.ct == 128)
    return v4 ? launch_gather<float, 4, 1>(a, d, L, w, SA, ldsa, Sb, sbs, st)
              : launch_gather<float, 1, 4>(a, d, L, w, SA, ldsa, Sb, sbs, st);
  return v4 ? launch_gather<float, 4, 2>(a, d, L, w, SA, ldsa, Sb, sbs, st)
            : launch_gather<float, 1, 8>(a, d, L, w, SA, ldsa, Sb, sbs, st);
}

sns_status cs_apply_dense_stream(const DenseArgs& a, int64_t d, uint64_t seed, void* SA, int64_t ldsa, void* Sb,
                                 int64_t sbs, cudaStream_t st) {
  // zero the outputs (row by row if strided)
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
  const bool v4 = (a.lda % 4 == 0) && (ldsa % 4 == 0) && (a.n % 4 == 0) && aligned(a.A, 16) && aligned(SA, 16);
  const uint64_t s0 = shift_state(stream_state(seed, kStreamCountSketch), a.row0);
  const int grid = num_sms() * 8;
  if (v4)
    {
      SNS_PROF(K_CS_STREAM, st);
    cs_stream_dense<4><<<grid, 256, 0, st>>>(static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b),
                                             a.m, a.n, (uint32_t)d, s0, static_cast<float*>(SA), ldsa,
                                             static_cast<float*>(Sb), sbs);
    }
  else
    {
      SNS_PROF(K_CS_STREAM, st);
    cs_stream_dense<1><<<grid, 256, 0, st>>>(static_cast<const float*>(a.A), a.lda, static_cast<const float*>(a.b),
                                             a.m, a.n, (uint32_t)d, s0, static_cast<float*>(SA), ldsa,
                                             static_cast<float*>(Sb), sbs);
    }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

int64_t cs_csr_sorted_max_n() { return (int64_t)(200 * 1024) / (4 * kGatherWarps) - 1; }

sns_status cs_apply_csr(const CsrArgs& a, int64_t d, uint64_t seed, float* SA, int64_t ldsa, float* Sb, int64_t sbs,
                        void* ws, size_t ws_bytes, cudaStream_t st) {
  if (a.n > cs_csr_sorted_max_n()) return SNS_EINVAL;
  const CsLayout L = cs_layout(a.m, a.n, d, false, true);
  if (ws_bytes < L.bytes) return SNS_ENOMEM;
  uint8_t* w = static_cast<uint8_t*>(ws);
  sns_status s = cs_phase1(a.m, d, seed, a.row0, L, w, st);
  if (s != SNS_OK) return s;
  const size_t smem = (size_t)kGatherWarps * (a.n + 1) * 4;     // one accumulator row per warp
  int dev = 0, smem_max = 0;
  SNS_CUDA_TRY(cudaGetDevice(&dev));
  SNS_CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)smem_max) return SNS_EINVAL;
  SNS_CUDA_TRY(raise_smem_limit((const void*)cs_gather_csr));
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cs_gather_csr, kGatherWarps * 32, smem));
  if (occ < 1) occ = 1;
  const int64_t items = d * L.parts;
  const int64_t grid = std::min<int64_t>(items, (int64_t)num_sms() * occ);
  {
    SNS_PROF(K_CS_CSR, st);
  cs_gather_csr<<<(unsigned)grid, kGatherWarps * 32, smem, st>>>(
      a.rowptr, a.col, a.val, a.b, a.n, (uint32_t)d, L.nblk, L.spi, L.parts,
      reinterpret_cast<const uint32_t*>(w + L.off_sorted), reinterpret_cast<const uint32_t*>(w + L.off_seg),
      reinterpret_cast<uint32_t*>(w + L.off_ticket), reinterpret_cast<float*>(w + L.off_part), SA, ldsa, Sb, sbs);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

// Streaming CountSketch on CSR: rows in order, chunks of 32 rows per warp
// (chunks go round the CTAs first), a lane per row with 8 entries loaded at
// once, rows with more than 32 nonzeros taken by the whole warp (16 entries per
// lane at once); every nonzero a_ij is added as s(i) a_ij into SA[h(i), j] by a
// float reduction in L2, b_i into Sb[h(i)].  One pass over the CSR arrays; the
// order of the additions into a given SA entry varies run to run.  SA and Sb
// must be zero.
constexpr int kCsrBatch = 8, kCsrLongBatch = 16, kCsrLongRow = 32;
__global__ void __launch_bounds__(256)
cs_stream_csr(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const float* __restrict__ val,
              const float* __restrict__ b, int64_t m, int64_t n, uint32_t d, uint64_t s0, float* __restrict__ SA,
              int64_t ldsa, float* __restrict__ Sb, int64_t sbs) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)w * gridDim.x + blockIdx.x;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = gw * 32; r0 < m; r0 += nw * 32) {
    const int64_t r = r0 + lane;
    int64_t e0 = 0, e1 = 0;
    uint32_t h = 0;
    float sg = 0.f;
    if (r < m) {
      e0 = __ldg(rowptr + r);
      e1 = __ldg(rowptr + r + 1);
      const uint64_t key = splitmix_at(s0, (uint64_t)r);
      h = bucket_of(key, d);
      sg = (key >> 63) ? -1.f : 1.f;
      atomicAdd(Sb + (int64_t)h * sbs, sg * __ldg(b + r));
    }
    const bool lng = (e1 - e0) > kCsrLongRow;
    if (!lng && r < m) {
      float* dst = SA + (int64_t)h * ldsa;
      for (int64_t eb = e0; eb < e1; eb += kCsrBatch) {
        int32_t cc[kCsrBatch];
        float vv[kCsrBatch];
#pragma unroll
        for (int u = 0; u < kCsrBatch; ++u) {
          const bool ok = eb + u < e1;
          cc[u] = ok ? __ldg(col + eb + u) : -1;
          vv[u] = ok ? __ldg(val + eb + u) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kCsrBatch; ++u)
          if ((uint32_t)cc[u] < (uint64_t)n) atomicAdd(dst + cc[u], sg * vv[u]);
      }
    }
    unsigned lm = __ballot_sync(0xffffffffu, lng);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int64_t a0 = __shfl_sync(0xffffffffu, e0, src), a1 = __shfl_sync(0xffffffffu, e1, src);
      const uint32_t hs = __shfl_sync(0xffffffffu, h, src);
      const float ss = __shfl_sync(0xffffffffu, sg, src);
      float* dst = SA + (int64_t)hs * ldsa;
      for (int64_t eb = a0; eb < a1; eb += 32 * kCsrLongBatch) {
        int32_t cc[kCsrLongBatch];
        float vv[kCsrLongBatch];
#pragma unroll
        for (int u = 0; u < kCsrLongBatch; ++u) {
          const int64_t e = eb + u * 32 + lane;
          cc[u] = e < a1 ? __ldg(col + e) : -1;
          vv[u] = e < a1 ? __ldg(val + e) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kCsrLongBatch; ++u)
          if ((uint32_t)cc[u] < (uint64_t)n) atomicAdd(dst + cc[u], ss * vv[u]);
      }
    }
  }
}

sns_status cs_apply_csr_stream(const CsrArgs& a, int64_t d, uint64_t seed, float* SA, int64_t ldsa, float* Sb,
                               int64_t sbs, cudaStream_t st) {
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
  int occ = 0;
  SNS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cs_stream_csr, 256, 0));
  const int grid = num_sms() * std::max(occ, 1);
  {
    SNS_PROF(K_CS_CSR, st);
    cs_stream_csr<<<grid, 256, 0, st>>>(a.rowptr, a.col, a.val, a.b, a.m, a.n, (uint32_t)d,
                                       shift_state(stream_state(seed, kStreamCountSketch), a.row0), SA, ldsa,
                                       Sb, sbs);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

sns_status cs_apply_sparse_sign(const DenseArgs& a, int64_t d, int zeta, uint64_t seed, float* SA, int64_t ldsa,
                                float* Sb, int64_t sbs, cudaStream_t st) {
  if (a.f64 || zeta < 1 || zeta > kSseMaxZeta || zeta > d) return SNS_EINVAL;
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
  const bool v4 = (a.lda % 4 == 0) && (ldsa % 4 == 0) && (a.n % 4 == 0) && aligned(a.A, 16) && aligned(SA, 16);
  // draw 0 of row i is output i of stream 0, draw z >= 1 output i (zeta - 1) + z - 1 of stream 4
  const uint64_t s0 = shift_state(stream_state(seed, kStreamCountSketch), a.row0);
  const uint64_t s4 = shift_state(stream_state(seed, kStreamSparseSign), (uint64_t)a.row0 * (uint64_t)(zeta - 1));
  const float scale = (float)(1.0 / std::sqrt((double)zeta));
  const int grid = num_sms() * 8;
  {
    SNS_PROF(K_CS_STREAM, st);
    if (v4)
      cs_sparse_sign_dense<4><<<grid, 256, 0, st>>>(static_cast<const float*>(a.A), a.lda,
                                                    static_cast<const float*>(a.b), a.m, a.n, (uint32_t)d, zeta, s0,
                                                    s4, scale, SA, ldsa, Sb, sbs);
    else
      cs_sparse_sign_dense<1><<<grid, 256, 0, st>>>(static_cast<const float*>(a.A), a.lda,
                                                    static_cast<const float*>(a.b), a.m, a.n, (uint32_t)d, zeta, s0,
                                                    s4, scale, SA, ldsa, Sb, sbs);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

int64_t cs_sorted_max_d() { return 8192; }

// Debug: buckets and signs of rows [0, m) exactly as the kernels compute them.
__global__ void cs_hash_dump(int64_t m, uint32_t d, uint64_t s0, uint32_t* h, int8_t* s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = splitmix_at(s0, (uint64_t)i);
    h[i] = bucket_of(key, d);
    s[i] = (key >> 63) ? -1 : 1;
  }
}
__global__ void stream_keys_dump(uint64_t s0, int64_t start, int64_t count, uint64_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = splitmix_at(s0, (uint64_t)(start + i));
}

sns_status debug_countsketch_hash(int64_t m, int64_t d, uint64_t seed, uint32_t* h, int8_t* s, cudaStream_t st) {
  {
    SNS_PROF(K_MISC, st);
  cs_hash_dump<<<num_sms() * 4, 256, 0, st>>>(m, (uint32_t)d, stream_state(seed, kStreamCountSketch), h, s);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}
sns_status debug_stream_keys(uint64_t seed, int stream, int64_t start, int64_t count, uint64_t* out, cudaStream_t st) {
  {
    SNS_PROF(K_MISC, st);
  stream_keys_dump<<<num_sms() * 4, 256, 0, st>>>(stream_state(seed, (uint64_t)stream), start, count, out);
  }
  SNS_LAUNCH_CHECK();
  return SNS_OK;
}

}  // namespace sns
