// segsplit.cuh -- device-wide split of the long segments of a segmented sort.
//
// A segment longer than the shared-memory capacity CAP cannot be sorted by one
// CTA in shared memory; one CTA takes it through global memory (an MSD pass,
// then its buckets in shared memory), which for a segment many times CAP long
// (a 567K-key segment of a lognormal batch) would outlast the rest of the
// batch.  Before the per-CTA sort runs, every segment above SPLIT_MIN_CAPS x CAP
// keys is cut into buckets by one stable MSD pass that all CTAs share, tile by
// tile:
//
//   split_classify_kernel  segments above SPLIT_MIN_CAPS x CAP keys go to the
//                          big list; the others (above one key) to the work
//                          list as they are
//   split_tiles_kernel     first tile of every big segment (exclusive scan of
//                          ceil(len / T)), total tile count
//   split_vary_kernel      per big segment, the OR of (radix key ^ radix key
//                          of its first element): the bits that vary in it
//   split_count_kernel     per tile, counts of the segment's split digit: the
//                          `bits` radix-key bits just below its highest
//                          varying bit, bits the smallest count that makes
//                          buckets average at most CAP / 2 (at most 8)
//   split_scan_kernel      per big segment, the offset of every (tile, digit)
//                          inside the segment (digit-major exclusive scan:
//                          stable), and one work item per non-empty bucket
//   split_scatter_kernel   per tile, a stable rank of its keys by digit (warp
//                          multisplit), staged in shared memory in digit order
//                          and written to the workspace copy in coalesced runs
//
// The digit is monotone in the radix key inside a segment (bits above the
// highest varying bit are equal), so sorting every bucket finishes the segment.
// The per-CTA kernel then takes the buckets (workspace copy -> keys) and the
// short segments (in place).  A big segment whose keys are all equivalent is
// already in order and gets no work at all.  Tile counts and tile ranges live
// in the device; the host launches persistent grids that read them, so the
// whole sequence is graph-capturable.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "segsort.cuh"

namespace ak {

// Bits of the split digit of a big segment and its shift.
__device__ __forceinline__ void split_digit_of(const BigSeg &b, int64_t cap, int &shift, uint32_t &mask) {
  const int hi = 63 - __clzll((long long)b.vary);
  const int lo = __ffsll((long long)b.vary) - 1;
  int bits = 1;
  while (bits < RADIX_BITS && (int64_t(cap / 2) << bits) < b.len) ++bits;
  shift = (hi - bits + 1) > lo ? (hi - bits + 1) : lo;
  mask = (1u << bits) - 1u;
}

// Big segment of split tile t: the last b with tile0 <= t.
__device__ __forceinline__ uint32_t split_find(const BigSeg *big, uint32_t nbig, uint32_t t) {
  uint32_t lo = 0, hi = nbig;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (big[mid].tile0 <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Segments above `split_min` keys go to the big list; the others (above one
// key) to the work list, those above `cap` (sorted by one CTA through global
// memory, the longest work) from its front, the rest from its back.
static __global__ void split_classify_kernel(const int64_t *off, int64_t nseg, int64_t n, int64_t cap,
                                             int64_t split_min, uint32_t *order, BigSeg *big, SplitState *st,
                                             const uint32_t *gate, uint32_t gate_want) {
  if (gate && *gate != gate_want) return;
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int64_t lo = off[s], hi = off[s + 1];
  lo = lo < 0 ? 0 : (lo > n ? n : lo);
  hi = hi < 0 ? 0 : (hi > n ? n : hi);
  const int64_t len = hi - lo;
  if (len > split_min) {
    const uint32_t b = atomicAdd(&st->nbig, 1u);
    big[b].lo = lo;
    big[b].len = len;
    big[b].vary = 0;
  } else if (len > cap) {
    order[atomicAdd(&st->nlong, 1u)] = uint32_t(s);
  } else if (len > 1) {
    order[nseg - 1 - atomicAdd(&st->nshort, 1u)] = uint32_t(s);
  }
}

// One CTA of 1024 threads: first tile of every big segment.
static __global__ void __launch_bounds__(1024) split_tiles_kernel(BigSeg *big, SplitState *st, int64_t tile,
                                                                  const uint32_t *gate, uint32_t gate_want) {
  if (gate && *gate != gate_want) return;
  __shared__ unsigned long long scr[1024 / 32 + 1];
  const uint32_t nbig = st->nbig;
  unsigned long long carry = 0;
  for (uint32_t c0 = 0; c0 < nbig; c0 += 1024) {
    const uint32_t b = c0 + threadIdx.x;
    const unsigned long long t = b < nbig ? (unsigned long long)((big[b].len + tile - 1) / tile) : 0ull;
    unsigned long long total;
    const unsigned long long ex = block_exclusive_scan<1024>(t, scr, &total);
    if (b < nbig) big[b].tile0 = uint32_t(carry + ex);
    carry += total;
  }
  if (threadIdx.x == 0) st->ntiles = uint32_t(carry);
}

template <typename U, int KIND>
__global__ void __launch_bounds__(SPLIT_BLOCK) split_vary_kernel(const U *keys, BigSeg *big, const SplitState *st,
                                                                 int64_t tile, U flip, const uint32_t *gate,
                                                                 uint32_t gate_want) {
  if (gate && *gate != gate_want) return;
  __shared__ unsigned long long scr[SPLIT_BLOCK / 32];
  const uint32_t nbig = st->nbig, ntiles = st->ntiles;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t b = split_find(big, nbig, t);
    const int64_t lo = big[b].lo, len = big[b].len;
    const int64_t t_lo = int64_t(t - big[b].tile0) * tile;
    const int64_t t_hi = (t_lo + tile) < len ? t_lo + tile : len;
    const U r0 = radix_key_t<KIND>(keys[lo], flip);
    unsigned long long v = 0;
    for (int64_t i = t_lo + threadIdx.x; i < t_hi; i += SPLIT_BLOCK)
      v |= (unsigned long long)U(radix_key_t<KIND>(keys[lo + i], flip) ^ r0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) scr[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long r = 0;
      for (int w = 0; w < SPLIT_BLOCK / 32; ++w) r |= scr[w];
      if (r) atomicOr(&big[b].vary, r);
    }
    __syncthreads();
  }
}

template <typename U, int KIND>
__global__ void __launch_bounds__(SPLIT_BLOCK) split_count_kernel(const U *keys, const BigSeg *big,
                                                                  const SplitState *st, int64_t tile, int64_t cap,
                                                                  U flip, uint32_t *tcount, const uint32_t *gate,
                                                                  uint32_t gate_want) {
  if (gate && *gate != gate_want) return;
  __shared__ uint32_t h[RADIX];
  const uint32_t nbig = st->nbig, ntiles = st->ntiles;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t b = split_find(big, nbig, t);
    const BigSeg bs = big[b];
    if (bs.vary == 0) continue;  // all keys equivalent: nothing to move (uniform over the CTA)
    int shift;
    uint32_t mask;
    split_digit_of(bs, cap, shift, mask);
    for (int i = threadIdx.x; i < RADIX; i += SPLIT_BLOCK) h[i] = 0u;
    __syncthreads();
    const int64_t t_lo = int64_t(t - bs.tile0) * tile;
    const int64_t t_hi = (t_lo + tile) < bs.len ? t_lo + tile : bs.len;
    for (int64_t i = t_lo + threadIdx.x; i < t_hi; i += SPLIT_BLOCK)
      atomicAdd(&h[uint32_t(radix_key_t<KIND>(keys[bs.lo + i], flip) >> shift) & mask], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < RADIX; i += SPLIT_BLOCK) tcount[size_t(t) * RADIX + i] = h[i];
    __syncthreads();
  }
}

// One CTA of RADIX threads per big segment (persistent over segments): turns
// the tile counts of the segment into offsets inside it and emits its buckets.
static __global__ void __launch_bounds__(RADIX) split_scan_kernel(const BigSeg *big, SplitState *st,
                                                                  uint32_t *tcount, BucketItem *buckets,
                                                                  const uint32_t *gate, uint32_t gate_want) {
  if (gate && *gate != gate_want) return;
  __shared__ unsigned long long scr[RADIX / 32 + 1];
  const uint32_t nbig = st->nbig;
  const uint32_t d = threadIdx.x;
  for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const BigSeg bs = big[b];
    if (bs.vary == 0) continue;
    const uint32_t t1 = (b + 1 < nbig) ? big[b + 1].tile0 : st->ntiles;
    uint32_t run = 0;
    for (uint32_t t = bs.tile0; t < t1; ++t) {
      const uint32_t c = tcount[size_t(t) * RADIX + d];
      tcount[size_t(t) * RADIX + d] = run;
      run += c;
    }
    unsigned long long total;
    const uint32_t start = uint32_t(block_exclusive_scan<RADIX>((unsigned long long)run, scr, &total));
    for (uint32_t t = bs.tile0; t < t1; ++t) tcount[size_t(t) * RADIX + d] += start;
    if (run > 0) {
      const uint32_t k = atomicAdd(&st->nbuck, 1u);
      buckets[k].lo = bs.lo + start;
      buckets[k].len = run;
    }
  }
}

// Stable scatter of every split tile into bucket order (workspace copy).
template <typename U, typename V, bool HAS_V, int KIND, int ITEMS>
struct SplitSmem {
  static constexpr int TILE = SPLIT_BLOCK * ITEMS;
  static constexpr int NW = SPLIT_BLOCK / 32;
  static constexpr int HSTRIDE = NW / 2 + 1;  // u32 words per digit row of per-warp u16 counters (odd)
  static constexpr int H2 = 2 * HSTRIDE;
  static constexpr int HROW = RADIX + 1;      // + the padding digit of a partial tile
  static constexpr size_t KEYS = size_t(TILE) * sizeof(U);
  static constexpr size_t VALS = HAS_V ? size_t(TILE) * sizeof(V) : 0;
  static constexpr size_t BUF = (KEYS + VALS + 127) / 128 * 128;
  static constexpr size_t OFF_OUT = BUF;                                          // tile in digit order
  static constexpr size_t OFF_HIST = 2 * BUF;                                     // u32[HROW][HSTRIDE]
  static constexpr size_t OFF_DIG = OFF_HIST + (size_t(HROW) * HSTRIDE * 4 + 15) / 16 * 16;  // u8[TILE]
  static constexpr size_t OFF_DST = OFF_DIG + (size_t(TILE) + 15) / 16 * 16;     // i64[RADIX]
  static constexpr size_t OFF_SCR = OFF_DST + RADIX * 8;                          // u32[RADIX/32]
  static constexpr size_t BYTES = OFF_SCR + 64;
  static_assert(TILE < 65536, "u16 warp bases");
};

template <typename U, typename V, bool HAS_V, int KIND, int ITEMS>
__global__ void __launch_bounds__(SPLIT_BLOCK, 2) split_scatter_kernel(const U *keys, const V *vals, U *alt_k, V *alt_v,
                                                                    const BigSeg *big, const SplitState *st,
                                                                    const uint32_t *tcount, int64_t cap, U flip,
                                                                    const uint32_t *gate, uint32_t gate_want) {
  using L = SplitSmem<U, V, HAS_V, KIND, ITEMS>;
  constexpr int TILE = L::TILE, NW = L::NW, H2 = L::H2, HROW = L::HROW;
  if (gate && *gate != gate_want) return;
  extern __shared__ __align__(128) uint8_t smem[];
  U *sk = reinterpret_cast<U *>(smem);
  V *sv = reinterpret_cast<V *>(smem + L::KEYS);
  U *ok = reinterpret_cast<U *>(smem + L::OFF_OUT);
  V *ov = reinterpret_cast<V *>(smem + L::OFF_OUT + L::KEYS);
  uint16_t *whist = reinterpret_cast<uint16_t *>(smem + L::OFF_HIST);
  uint32_t *whist32 = reinterpret_cast<uint32_t *>(smem + L::OFF_HIST);
  uint8_t *s_dig = smem + L::OFF_DIG;
  long long *s_dst = reinterpret_cast<long long *>(smem + L::OFF_DST);
  uint32_t *s_scr = reinterpret_cast<uint32_t *>(smem + L::OFF_SCR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t lt_mask = lanemask_lt();
  const uint32_t gt_mask = ~(lt_mask | (1u << lane));
  const uint32_t nbig = st->nbig, ntiles = st->ntiles;
  for (int i = tid; i < HROW * L::HSTRIDE; i += SPLIT_BLOCK) whist32[i] = 0u;
  __syncthreads();
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint32_t b = split_find(big, nbig, t);
    const BigSeg bs = big[b];
    if (bs.vary == 0) continue;  // uniform over the CTA
    int shift;
    uint32_t mask;
    split_digit_of(bs, cap, shift, mask);
    const int64_t t_lo = int64_t(t - bs.tile0) * TILE;
    const int tile_n = int((bs.len - t_lo) < int64_t(TILE) ? (bs.len - t_lo) : int64_t(TILE));
    const U *gk = keys + bs.lo + t_lo;
    const V *gv = HAS_V ? vals + bs.lo + t_lo : nullptr;
    for (int i = tid; i < tile_n; i += SPLIT_BLOCK) {
      sk[i] = gk[i];
      if (HAS_V) sv[i] = gv[i];
    }
    __syncthreads();  // A: tile staged
    // ---- warp multisplit rank (item i of lane l at wbase + 32 i + l)
    const int wbase = warp * 32 * ITEMS;
    uint32_t dr[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int idx = wbase + i * 32 + lane;
      dr[i] = idx < tile_n ? (uint32_t(radix_key_t<KIND>(sk[idx], flip) >> shift) & mask) : uint32_t(RADIX);
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t d = dr[i];
      uint32_t peers = __ballot_sync(0xffffffffu, d < uint32_t(RADIX));
      if (d >= uint32_t(RADIX)) peers = ~peers;
#pragma unroll
      for (int bit = 0; bit < RADIX_BITS; ++bit) {
        const bool on = (d >> bit) & 1u;
        const uint32_t v = __ballot_sync(0xffffffffu, on);
        peers &= on ? v : ~v;
      }
      uint16_t *wc = whist + d * H2 + warp;
      const uint32_t cnt = *wc;
      __syncwarp();
      if ((peers & gt_mask) == 0) *wc = uint16_t(cnt + __popc(peers));
      __syncwarp();
      dr[i] = ((cnt + __popc(peers & lt_mask)) << 9) | d;
    }
    __syncthreads();  // B: warp counters complete
    uint32_t my = 0, inc = 0;
    uint32_t *hrow = whist32 + tid * L::HSTRIDE;
    if (tid < RADIX) {
#pragma unroll
      for (int v = 0; v < NW / 2; ++v) {
        const uint32_t w = hrow[v];
        my += (w & 0xFFFFu) + (w >> 16);
      }
      inc = warp_inclusive_scan(my);
      if (lane == 31) s_scr[warp] = inc;
    }
    __syncthreads();  // C: warp totals
    if (tid < RADIX) {
      uint32_t start = inc - my;
#pragma unroll
      for (int w2 = 0; w2 < RADIX / 32; ++w2)
        if (w2 < warp) start += s_scr[w2];
      uint32_t run = start;
#pragma unroll
      for (int v = 0; v < NW / 2; ++v) {
        const uint32_t w = hrow[v];
        const uint32_t lo = run, hi = run + (w & 0xFFFFu);
        run = hi + (w >> 16);
        hrow[v] = (lo & 0xFFFFu) | (hi << 16);
      }
      // destination of this tile's first slot of digit tid, in the copy
      s_dst[tid] = (long long)(bs.lo + tcount[size_t(t) * RADIX + tid]) - (long long)start;
    }
    __syncthreads();  // D: warp bases, destinations
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t d = dr[i] & 511u;
      if (d < uint32_t(RADIX)) {
        const int idx = wbase + i * 32 + lane;
        const uint32_t pos = uint32_t(whist[d * H2 + warp]) + (dr[i] >> 9);
        ok[pos] = sk[idx];
        if (HAS_V) ov[pos] = sv[idx];
        s_dig[pos] = uint8_t(d);
      }
    }
    __syncthreads();  // E: tile in digit order
    for (int i = tid; i < HROW * L::HSTRIDE; i += SPLIT_BLOCK) whist32[i] = 0u;
    for (int i = tid; i < tile_n; i += SPLIT_BLOCK) {
      const long long dst = s_dst[s_dig[i]] + i;
      alt_k[dst] = ok[i];
      if (HAS_V) alt_v[dst] = ov[i];
    }
    __syncthreads();  // F: buffers free for the next tile
  }
}

}  // namespace ak
