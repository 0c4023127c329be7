// segsort.cuh -- segmented sort: many independent CSR segments in one
// persistent launch (and the one-launch small-n sort, a single segment).
//
// classify_kernel  builds the work order: segments above the shared-memory
//                  capacity first (they take longest), then the rest (with
//                  the device-wide split of segsplit.cuh, its classifier
//                  builds the order instead)
// segsort_kernel   persistent CTAs pop work items from a device work counter.
//   * L <= CAP: the segment is loaded into shared memory and its radix-key
//     range [rmin, rmax] found in the same pass.  One counting pass spreads
//     the keys over up to 2^SUB_BITS sub-ranges of equal width
//     ((r - rmin) >> sh, monotone in r; a key or two each when the keys are
//     spread smoothly); 16-bit input positions are scattered by sub-range;
//     then every key counts the keys of its own sub-range that come before it
//     in (radix key, input position) order -- which keeps the sort stable --
//     and is written straight to its output slot.  When a sub-range holds more
//     than SUB_MAX keys
//     (clustered keys), the segment instead takes stable LSD passes over only
//     the radix bits that vary inside it (OR of r ^ r0), through a global
//     workspace copy, chunk by chunk with warp ranks.
//   * L > CAP: one stable MSD pass through global memory on the top varying
//     bits (just enough that buckets average CAP/2 keys; workspace copy of the
//     segment), then each bucket is sorted in shared memory like a small
//     segment -- or, if a bucket is still above CAP, by chunked LSD passes
//     through global memory.
// Every pass is stable, so every segment ends in the stable order of the key
// transform of common.cuh.  Raw key bits (and values) are moved.
#pragma once

#include "common.cuh"

namespace ak {

constexpr int SUB_BITS = 12;  // at most 2^SUB_BITS sub-ranges per segment
constexpr int SUB_MAX = 48;   // largest sub-range a segment sorts by counting (else LSD passes)
// sub-ranges per segment about len / 2^AK_SUB_SLACK (at most 2^SUB_BITS)
#ifndef AK_SUB_SLACK
#define AK_SUB_SLACK 1
#endif

struct SplitState {  // zeroed by the caller
  uint32_t nbig;     // big segments (split across CTAs)
  uint32_t nlong;    // segments above the shared capacity, sorted by one CTA (front of the work list)
  uint32_t nshort;   // segments within the shared capacity (back of the work list)
  uint32_t nbuck;    // bucket work items of the big segments
  uint32_t ntiles;   // split tiles over all big segments
  uint32_t pad[3];
};

struct BigSeg {
  int64_t lo, len;              // key range [lo, lo + len)
  unsigned long long vary;      // OR of (radix key ^ radix key of keys[lo])
  uint32_t tile0;               // first split tile
  uint32_t pad;
};

struct BucketItem {
  int64_t lo, len;  // [lo, lo + len) in the workspace copy; sorted into the keys
};
static_assert(sizeof(BigSeg) == 32 && sizeof(BucketItem) == 16, "workspace sizes of the split tables");


struct SegArgsBase {
  const int64_t *off;     // nseg + 1 offsets (clamped to [0, n] on read); NULL: tiles of tile_len
  int64_t tile_len;       // off == NULL: segment s = [s * tile_len, (s + 1) * tile_len) within [0, n)
  int64_t nseg;
  int64_t n;
  const uint32_t *order;  // work order (segment ids), nseg entries (NULL with off == NULL)
  DevHeader *hdr;
  int path_tag;           // written to ak_info.path by block 0
  const uint32_t *gate;   // if set, run only when *gate == gate_want
  uint32_t gate_want;
  // device-wide split (segsplit.cuh): work items are the buckets of the long
  // segments (workspace copy -> keys), then the short segments of `order`
  const SplitState *split;
  const BucketItem *buckets;
};

template <typename U, typename V>
struct SegArgs : SegArgsBase {
  U *keys;     // in place
  V *vals;     // in place (HAS_V)
  U *alt_k;    // workspace copy region, indexed like keys
  V *alt_v;
  U flip;
  int64_t seg_base;  // added to every offset (0 for the batch API)
};

// ------------------------------------------------------------- classification
// Work order: segments longer than `cap` from the front, the others from the back.
static __global__ void classify_kernel(const int64_t *off, int64_t nseg, int64_t n, int64_t cap, uint32_t *order,
                                       uint32_t *counters, const uint32_t *gate, uint32_t gate_want) {
  if (gate && *gate != gate_want) return;
  const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= nseg) return;
  int64_t lo = off[s], hi = off[s + 1];
  lo = lo < 0 ? 0 : (lo > n ? n : lo);
  hi = hi < 0 ? 0 : (hi > n ? n : hi);
  if (hi - lo > cap) order[atomicAdd(&counters[0], 1u)] = uint32_t(s);
  else order[nseg - 1 - atomicAdd(&counters[1], 1u)] = uint32_t(s);
}

// Clamp an offset into [0, n].
__device__ __forceinline__ int64_t clamp_off(int64_t v, int64_t n) { return v < 0 ? 0 : (v > n ? n : v); }

// Reduction helpers over the CTA.
template <int BLOCK>
__device__ __forceinline__ unsigned long long cta_or(unsigned long long v, unsigned long long *scr) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) scr[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = 0;
#pragma unroll
  for (int w = 0; w < BLOCK / 32; ++w) r |= scr[w];
  __syncthreads();
  return r;
}

template <typename U, typename V, bool HAS_V, int KIND, int BLOCK, int ITEMS, int CAP>
struct SegSmem {
  static constexpr int NW = BLOCK / 32;
  static constexpr int CH = BLOCK * ITEMS;  // keys ranked per chunk
  static constexpr int HROW = RADIX + 2;
  // buffer A: CAP keys, then (16-byte aligned) CAP values; buffer B: CAP
  // 16-bit input positions
  static constexpr size_t VOFF = (size_t(CAP) * sizeof(U) + 15) / 16 * 16;
  static constexpr size_t BUF = (VOFF + (HAS_V ? size_t(CAP) * sizeof(V) : 0) + 127) / 128 * 128;
  static constexpr size_t OFF_A = 0;
  static constexpr size_t OFF_B = BUF;
  static constexpr size_t OFF_HIST = BUF + (size_t(CAP) * 2 + 127) / 128 * 128;      // u16[NW][HROW]
  static constexpr size_t OFF_MASK = (OFF_HIST + size_t(NW) * HROW * 2 + 15) / 16 * 16;  // u32[NW][HROW]
  static constexpr size_t OFF_CNT = OFF_MASK + size_t(NW) * HROW * 4;               // u32[RADIX] digit hist
  static constexpr size_t OFF_RUN = OFF_CNT + RADIX * 4;                            // u32[RADIX] running offsets
  static constexpr size_t OFF_CST = OFF_RUN + RADIX * 4;                            // u32[RADIX] chunk starts
  static constexpr size_t OFF_CCNT = OFF_CST + RADIX * 4;                           // u32[RADIX] chunk counts
  static constexpr size_t OFF_BST = OFF_CCNT + RADIX * 4;                           // u32[RADIX] bucket starts
  static constexpr size_t OFF_BCNT = OFF_BST + RADIX * 4;                           // u32[RADIX] bucket counts
  static constexpr size_t OFF_SCR = OFF_BCNT + RADIX * 4;                           // u64[NW+1]
  static constexpr size_t OFF_MISC = OFF_SCR + (NW + 1) * 8;                        // u32[8 + NW]
  static constexpr size_t BYTES = OFF_MISC + (8 + NW) * 4;
  static_assert(CH <= CAP, "a chunk fits in a segment buffer");
  static_assert(VOFF % 16 == 0 && BUF % 128 == 0 && OFF_MASK % 16 == 0 && OFF_SCR % 8 == 0,
                "shared-memory arrays aligned to their element size");
  static_assert(CAP < 65536, "16-bit warp bases and input positions");
  static_assert(size_t(NW) * HROW * 4 >= (size_t(1) << SUB_BITS) * 4, "sub-range counters fit in the mask words");
};

// One CTA sorts segments.  Generic pointers address shared or global buffers.
template <typename U, typename V, bool HAS_V, int KIND, int BLOCK, int ITEMS, int CAP>
struct SegCta {
  using L = SegSmem<U, V, HAS_V, KIND, BLOCK, ITEMS, CAP>;
  static constexpr int NW = L::NW, CH = L::CH, HROW = L::HROW;
  uint8_t *smem;
  int tid, warp, lane;
  uint32_t lt_mask, gt_mask;
  U flip;
  uint16_t *whist, *wh;
  uint32_t *wmask, *wm, *s_cnt, *s_run, *s_cst, *s_ccnt, *s_bst, *s_bcnt, *s_misc;
  unsigned long long *s_scr;

  __device__ void init(uint8_t *sm, U fl) {
    smem = sm;
    tid = threadIdx.x;
    warp = tid >> 5;
    lane = tid & 31;
    lt_mask = lanemask_lt();
    gt_mask = ~(lt_mask | (1u << lane));
    flip = fl;
    whist = reinterpret_cast<uint16_t *>(smem + L::OFF_HIST);
    wh = whist + warp * HROW;
    wmask = reinterpret_cast<uint32_t *>(smem + L::OFF_MASK);
    wm = wmask + warp * HROW;
    s_cnt = reinterpret_cast<uint32_t *>(smem + L::OFF_CNT);
    s_run = reinterpret_cast<uint32_t *>(smem + L::OFF_RUN);
    s_cst = reinterpret_cast<uint32_t *>(smem + L::OFF_CST);
    s_ccnt = reinterpret_cast<uint32_t *>(smem + L::OFF_CCNT);
    s_bst = reinterpret_cast<uint32_t *>(smem + L::OFF_BST);
    s_bcnt = reinterpret_cast<uint32_t *>(smem + L::OFF_BCNT);
    s_scr = reinterpret_cast<unsigned long long *>(smem + L::OFF_SCR);
    s_misc = reinterpret_cast<uint32_t *>(smem + L::OFF_MISC);
    for (int i = tid; i < NW * HROW; i += BLOCK) wmask[i] = 0u;
    __syncthreads();
  }

  __device__ U *buf_k(int which) { return reinterpret_cast<U *>(smem + (which ? L::OFF_B : L::OFF_A)); }
  __device__ V *buf_v(int which) { return reinterpret_cast<V *>(smem + (which ? L::OFF_B : L::OFF_A) + L::VOFF); }
  __device__ U rk(U k) const { return radix_key_t<KIND>(k, flip); }

  // OR over the segment of (radix key ^ radix key of the first element).
  __device__ unsigned long long vary_bits(const U *src, int64_t len) {
    const U r0 = rk(src[0]);
    unsigned long long v = 0;
    for (int64_t i = tid; i < len; i += BLOCK) v |= (unsigned long long)(rk(src[i]) ^ r0);
    return cta_or<BLOCK>(v, s_scr);
  }

  // Copy len elements (keys and values) between generic buffers, coalesced.
  __device__ void copy(U *dk, V *dv, const U *sk, const V *sv, int64_t len) {
    for (int64_t i = tid; i < len; i += BLOCK) {
      dk[i] = sk[i];
      if (HAS_V) dv[i] = sv[i];
    }
  }

  // Rank one chunk [c0, c0 + cn) of src by digit (shift) with warp multisplit;
  // afterwards wh rows hold chunk digit start + earlier-warp counts, s_cst the
  // chunk digit starts and s_ccnt the chunk digit counts.
  __device__ void rank_chunk(const U *src, int cn, int shift, uint32_t (&dr)[ITEMS]) {
    for (int i = lane; i < HROW / 2; i += 32) reinterpret_cast<uint32_t *>(wh)[i] = 0u;
    __syncwarp();
    const int wbase = warp * 32 * ITEMS;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int idx = wbase + i * 32 + lane;
      dr[i] = (idx < cn) ? digit_of(rk(src[idx]), shift) : uint32_t(RADIX);
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t d = dr[i];
      atomicOr(&wm[d], 1u << lane);
      __syncwarp();
      const uint32_t peers = wm[d];
      const uint32_t cnt = wh[d];
      __syncwarp();
      if ((peers & gt_mask) == 0) {
        wh[d] = uint16_t(cnt + __popc(peers));
        wm[d] = 0u;
      }
      __syncwarp();
      dr[i] = ((cnt + __popc(peers & lt_mask)) << 9) | d;
    }
    __syncthreads();
    uint32_t my = 0;
    if (tid < RADIX) {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = whist[w * HROW + tid];
        whist[w * HROW + tid] = uint16_t(run);
        run += c;
      }
      my = run;
      s_ccnt[tid] = run;
    }
    unsigned long long total;
    const uint32_t start =
        uint32_t(block_exclusive_scan<BLOCK>((unsigned long long)(tid < RADIX ? my : 0u), s_scr, &total));
    if (tid < RADIX) {
      s_cst[tid] = start;
#pragma unroll
      for (int w = 0; w < NW; ++w) whist[w * HROW + tid] = uint16_t(whist[w * HROW + tid] + start);
    }
    __syncthreads();
  }

  // Digit histogram of src[0, len) into s_cnt, exclusive scan into s_run.
  __device__ void digit_offsets(const U *src, int64_t len, int shift) {
    for (int i = tid; i < RADIX; i += BLOCK) s_cnt[i] = 0u;
    __syncthreads();
    for (int64_t i = tid; i < len; i += BLOCK) atomicAdd(&s_cnt[digit_of(rk(src[i]), shift)], 1u);
    __syncthreads();
    unsigned long long total;
    const uint32_t c = tid < RADIX ? s_cnt[tid] : 0u;
    const uint32_t ex = uint32_t(block_exclusive_scan<BLOCK>((unsigned long long)c, s_scr, &total));
    if (tid < RADIX) s_run[tid] = ex;
    __syncthreads();
  }

  // One stable pass src -> dst in global memory (len > CAP possible), chunks
  // staged through buffer A so that every warp stores digit runs.  If
  // `buckets`, s_bst/s_bcnt receive the digit starts/counts.
  __device__ void pass_global(const U *sk, const V *sv, U *dk, V *dv, int64_t len, int shift, bool buckets) {
    for (int i = tid; i < NW * HROW; i += BLOCK) wmask[i] = 0u;  // ranking state (sort_small leaves counters)
    digit_offsets(sk, len, shift);
    if (buckets && tid < RADIX) {
      s_bst[tid] = s_run[tid];
      s_bcnt[tid] = s_cnt[tid];
    }
    U *stk = buf_k(0);
    V *stv = buf_v(0);
    for (int64_t c0 = 0; c0 < len; c0 += CH) {
      const int cn = int((len - c0) < CH ? (len - c0) : CH);
      uint32_t dr[ITEMS];
      rank_chunk(sk + c0, cn, shift, dr);
      const int wbase = warp * 32 * ITEMS;
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const uint32_t d = dr[i] & 511u;
        if (d < RADIX) {
          const int idx = wbase + i * 32 + lane;
          const uint32_t pos = uint32_t(wh[d]) + (dr[i] >> 9);
          stk[pos] = sk[c0 + idx];
          if (HAS_V) stv[pos] = sv[c0 + idx];
        }
      }
      __syncthreads();
      for (int i = tid; i < cn; i += BLOCK) {
        const U k = stk[i];
        const uint32_t d = digit_of(rk(k), shift);
        const int64_t g = int64_t(s_run[d]) + (i - int64_t(s_cst[d]));
        dk[g] = k;
        if (HAS_V) dv[g] = stv[i];
      }
      __syncthreads();
      if (tid < RADIX) s_run[tid] += s_ccnt[tid];
      __syncthreads();
    }
  }

  // Range of the radix keys of a shared buffer: min, max and OR of (r ^ r[0]).
  __device__ void key_range(const U *src, int len, U &mn, U &mx, unsigned long long &vary) {
    const U r0 = rk(src[0]);
    U lo = r0, hi = r0;
    unsigned long long v = 0;
    for (int i = tid; i < len; i += BLOCK) {
      const U r = rk(src[i]);
      lo = r < lo ? r : lo;
      hi = r > hi ? r : hi;
      v |= (unsigned long long)(U(r ^ r0));
    }
    unsigned long long l64 = lo, h64 = hi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, l64, o);
      const unsigned long long hi2 = __shfl_xor_sync(0xffffffffu, h64, o);
      v |= __shfl_xor_sync(0xffffffffu, v, o);
      l64 = lo2 < l64 ? lo2 : l64;
      h64 = hi2 > h64 ? hi2 : h64;
    }
    unsigned long long *scr = reinterpret_cast<unsigned long long *>(s_cnt);  // 3 x NW words
    if (lane == 0) {
      scr[warp] = l64;
      scr[NW + warp] = h64;
      scr[2 * NW + warp] = v;
    }
    __syncthreads();
    l64 = scr[0];
    h64 = scr[NW];
    v = scr[2 * NW];
#pragma unroll
    for (int w = 1; w < NW; ++w) {
      l64 = scr[w] < l64 ? scr[w] : l64;
      h64 = scr[NW + w] > h64 ? scr[NW + w] : h64;
      v |= scr[2 * NW + w];
    }
    __syncthreads();
    mn = U(l64);
    mx = U(h64);
    vary = v;
  }

  // Exclusive scan of cnt[0, m) in place; returns the largest count.
  __device__ uint32_t scan_counts(uint32_t *cnt, int m) {
    const int per = (m + BLOCK - 1) / BLOCK;
    const int b0 = tid * per, b1 = (b0 + per) < m ? (b0 + per) : m;
    uint32_t sum = 0, big = 0;
    for (int i = b0; i < b1; ++i) {
      const uint32_t c = cnt[i];
      sum += c;
      big = c > big ? c : big;
    }
    unsigned long long total;
    uint32_t run = uint32_t(block_exclusive_scan<BLOCK>((unsigned long long)sum, s_scr, &total));
    for (int i = b0; i < b1; ++i) {
      const uint32_t c = cnt[i];
      cnt[i] = run;
      run += c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t b2 = __shfl_xor_sync(0xffffffffu, big, o);
      big = b2 > big ? b2 : big;
    }
    uint32_t *wbig = s_misc + 8;  // one word per warp
    if (lane == 0) wbig[warp] = big;
    __syncthreads();
    big = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) big = wbig[w] > big ? wbig[w] : big;
    __syncthreads();
    return big;
  }

  // Sort gk/gv[0, len) (global) into dk/dv (global, may alias gk/gv), len <= CAP;
  // tk/tv: len elements of global scratch other than dk/dv (may alias gk/gv).
  // Five CTA barriers; the caller separates consecutive calls by a barrier.
  __device__ void sort_small(const U *gk, const V *gv, U *dk, V *dv, int len, U *tk, V *tv) {
    // radix-key arithmetic in 32 bits for keys of 32 bits or less
    using R = typename std::conditional<(sizeof(U) <= 4), uint32_t, unsigned long long>::type;
    U *ak = buf_k(0);
    V *av = buf_v(0);
    // 1. load into shared memory with the range of the radix keys: min, max and
    //    OR of (r ^ r of the first key), reduced per warp, then by every warp
    //    over the warp partials
    R *scr = reinterpret_cast<R *>(s_cnt);  // 3 x NW partials
    uint32_t *sub = wmask;                   // sub-range counters, cleared here for this segment
    for (int i = tid; i < (1 << SUB_BITS); i += BLOCK) sub[i] = 0u;
    const R r0 = R(rk(gk[0]));
    R lo = R(~R(0)), hi = 0, vary = 0;
    auto stage = [&](int i, U k) {
      ak[i] = k;
      const R r = R(rk(k));
      lo = r < lo ? r : lo;
      hi = r > hi ? r : hi;
      vary |= r ^ r0;
    };
    int i0 = tid;
    for (; i0 + 3 * BLOCK < len; i0 += 4 * BLOCK) {  // four loads in flight before the stores
      const U k0 = gk[i0], k1 = gk[i0 + BLOCK], k2 = gk[i0 + 2 * BLOCK], k3 = gk[i0 + 3 * BLOCK];
      stage(i0, k0);
      stage(i0 + BLOCK, k1);
      stage(i0 + 2 * BLOCK, k2);
      stage(i0 + 3 * BLOCK, k3);
    }
    for (; i0 < len; i0 += BLOCK) stage(i0, gk[i0]);
    if (HAS_V)
      for (int i = tid; i < len; i += BLOCK) av[i] = gv[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const R l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
      vary |= __shfl_xor_sync(0xffffffffu, vary, o);
      lo = l2 < lo ? l2 : lo;
      hi = h2 > hi ? h2 : hi;
    }
    if (lane == 0) {
      scr[warp] = lo;
      scr[NW + warp] = hi;
      scr[2 * NW + warp] = vary;
    }
    __syncthreads();  // [1] keys staged, warp partials written
    lo = lane < NW ? scr[lane] : R(~R(0));
    hi = lane < NW ? scr[NW + lane] : R(0);
    vary = lane < NW ? scr[2 * NW + lane] : R(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const R l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
      vary |= __shfl_xor_sync(0xffffffffu, vary, o);
      lo = l2 < lo ? l2 : lo;
      hi = h2 > hi ? h2 : hi;
    }
    if (vary == 0) {  // every key equivalent: stable order is the input order
      if (dk != gk) copy(dk, dv, ak, av, len);
      return;
    }
    // 2. sub-ranges of width 2^sh over [lo, hi]: about two keys each when the
    //    keys are spread evenly; counts in the (zero) mask words
    const R span = R(hi - lo);
    const int span_bits = sizeof(R) == 4 ? 32 - __clz(uint32_t(span)) : 64 - __clzll((long long)span);
    int want = (32 - __clz(uint32_t(len - 1))) - AK_SUB_SLACK;
    want = want < 1 ? 1 : (want > SUB_BITS ? SUB_BITS : want);
    const int sh = span_bits > want ? span_bits - want : 0;
    const int nsub = int(span >> sh) + 1;
    for (int i = tid; i < len; i += BLOCK) atomicAdd(&sub[R(R(rk(ak[i])) - lo) >> sh], 1u);
    __syncthreads();  // [2] counts complete
    // 3. exclusive scan of the counts and the largest count: per-thread runs of
    //    counters, warp scans, every warp combines the warp totals itself
    uint32_t *scr32 = s_cnt + 8 * NW;  // words of their own, past the range partials
    const int per = (nsub + BLOCK - 1) / BLOCK;
    const int b0 = tid * per, b1 = (b0 + per) < nsub ? (b0 + per) : nsub;
    uint32_t sum = 0, big = 0;
    for (int i = b0; i < b1; ++i) {
      const uint32_t c = sub[i];
      sum += c;
      big = c > big ? c : big;
    }
    const uint32_t winc = warp_inclusive_scan(sum);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t b2 = __shfl_xor_sync(0xffffffffu, big, o);
      big = b2 > big ? b2 : big;
    }
    if (lane == 31) scr32[warp] = winc;
    if (lane == 0) scr32[NW + warp] = big;
    __syncthreads();  // [3] warp totals
    {
      const uint32_t t = lane < NW ? scr32[lane] : 0u;
      const uint32_t tinc = warp_inclusive_scan(t);
      const uint32_t wbase = __shfl_sync(0xffffffffu, tinc - t, warp);
      big = lane < NW ? scr32[NW + lane] : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const uint32_t b2 = __shfl_xor_sync(0xffffffffu, big, o);
        big = b2 > big ? b2 : big;
      }
      uint32_t run = wbase + winc - sum;
      for (int i = b0; i < b1; ++i) {
        const uint32_t c = sub[i];
        sub[i] = run;
        run += c;
      }
    }
    __syncthreads();  // [4] offsets in place
    if (big > uint32_t(SUB_MAX)) {  // clustered keys: LSD over the varying bits
      for (int i = tid; i < nsub; i += BLOCK) sub[i] = 0u;
      copy(tk, tv, ak, av, len);  // buffer A stages the chunks of the passes
      __syncthreads();
      const int vlo = __ffsll((long long)vary) - 1;
      const int vhi = 63 - __clzll((long long)vary);
      lsd_global(tk, tv, dk, dv, len, vlo, vhi, dk, dv);
      return;
    }
    // 4. input positions by sub-range (any order inside a sub-range) ...
    uint16_t *pos = reinterpret_cast<uint16_t *>(buf_k(1));
    for (int i = tid; i < len; i += BLOCK) {
      const uint32_t slot = atomicAdd(&sub[R(R(rk(ak[i])) - lo) >> sh], 1u);
      pos[slot] = uint16_t(i);
    }
    __syncthreads();  // [5] sub[s] now holds the end of sub-range s
    // 5. ... then every key finds its place in its sub-range by counting the
    //    keys there that come before it in (radix key, input position) order
    //    (independent loads: no chain of dependent moves), and goes straight to
    //    its output slot.  The counters stay as they are: the next segment
    //    clears them, and pass_global clears them before it ranks.
    for (int j = tid; j < len; j += BLOCK) {
      const int x = pos[j];
      const U kx = ak[x];
      const R rx = R(rk(kx));
      const uint32_t s_ = uint32_t(R(rx - lo) >> sh);
      const int b = s_ ? int(sub[s_ - 1]) : 0, e = int(sub[s_]);
      int rank = 0;
      for (int i = b; i < e; ++i) {
        const int y = pos[i];
        const R ry = R(rk(ak[y]));
        rank += (ry < rx || (ry == rx && y < x)) ? 1 : 0;
      }
      dk[b + rank] = kx;
      if (HAS_V) dv[b + rank] = av[x];
    }
  }

  // Chunked LSD through global memory over bits [lo, hi]: src -> alternating
  // buffers, result left in dk/dv.
  __device__ void lsd_global(U *k0, V *v0, U *k1, V *v1, int64_t len, int lo, int hi, U *dk, V *dv) {
    // k0 holds the data; passes alternate k0 -> k1 -> k0 ...
    int which = 0;
    for (int sh = lo; sh <= hi; sh += RADIX_BITS) {
      if (which == 0) pass_global(k0, v0, k1, v1, len, sh, false);
      else pass_global(k1, v1, k0, v0, len, sh, false);
      which ^= 1;
    }
    U *rk_ = which ? k1 : k0;
    V *rv_ = which ? v1 : v0;
    if (rk_ != dk) {
      copy(dk, dv, rk_, rv_, len);
      __syncthreads();
    }
  }

  // Segment above CAP: one stable MSD split on the top varying bits -- just
  // enough of them that buckets average about CAP/2 keys -- then every bucket
  // is sorted in shared memory (or, if still above CAP, by chunked passes
  // through global memory).
  __device__ void sort_large(U *gk, V *gv, U *ak, V *av, int64_t len) {
    const unsigned long long vary = vary_bits(gk, len);
    if (vary == 0) return;
    const int lo = __ffsll((long long)vary) - 1;
    const int hi = 63 - __clzll((long long)vary);
    int bits = 1;
    while (bits < RADIX_BITS && (int64_t(CAP / 2) << bits) < len) ++bits;
    const int top = (hi - bits + 1) > lo ? (hi - bits + 1) : lo;
    // digit = (r >> top) & 255: bits above hi are constant, so only 2^(hi-top+1) buckets occur
    pass_global(gk, gv, ak, av, len, top, true);  // keys now in ak in top-digit order
    if (top == lo) {  // that pass covered every varying bit
      copy(gk, gv, ak, av, len);
      __syncthreads();
      return;
    }
    for (int b = 0; b < RADIX; ++b) {
      const int64_t bs = s_bst[b], bl = s_bcnt[b];
      if (bl == 0) continue;
      if (bl <= CAP) {
        sort_small(ak + bs, HAS_V ? av + bs : nullptr, gk + bs, HAS_V ? gv + bs : nullptr, int(bl), ak + bs,
                   HAS_V ? av + bs : nullptr);
        __syncthreads();  // the next bucket reuses the shared buffers
      } else {
        // still too large: chunked LSD over the bits below the top digit
        const unsigned long long bv = vary_bits(ak + bs, bl);
        if (bv == 0) {
          copy(gk + bs, HAS_V ? gv + bs : nullptr, ak + bs, HAS_V ? av + bs : nullptr, bl);
          __syncthreads();
          continue;
        }
        const int blo = __ffsll((long long)bv) - 1;
        const int bhi = 63 - __clzll((long long)bv);
        lsd_global(ak + bs, HAS_V ? av + bs : nullptr, gk + bs, HAS_V ? gv + bs : nullptr, bl, blo, bhi,
                   gk + bs, HAS_V ? gv + bs : nullptr);
      }
    }
  }
};

// Two CTAs per SM: the register cap (64) spills a few hundred bytes in the
// kernels with values, and still beats one CTA per SM at their ~100 registers
// (learned sortperm / pairs of 2^28 int64 keys 5-10% faster, keys-only 14%).
template <typename U, typename V, bool HAS_V, int KIND, int BLOCK, int ITEMS, int CAP>
__global__ void __launch_bounds__(BLOCK, 2) segsort_kernel(SegArgs<U, V> a) {
  using C = SegCta<U, V, HAS_V, KIND, BLOCK, ITEMS, CAP>;
  if (a.gate && *a.gate != a.gate_want) return;
  extern __shared__ __align__(128) uint8_t smem[];
  C c;
  c.init(smem, a.flip);
  uint32_t *s_work = c.s_misc;
  if (blockIdx.x == 0 && c.tid == 0 && a.path_tag) a.hdr->info.path = a.path_tag;
  // with the split, work items are: the long segments (one CTA each, through
  // global memory), the buckets of the big ones, the short segments -- longest
  // work first
  int64_t nlong = 0, nbuck = 0, nshort = 0, nwork = a.nseg;
  if (a.split) {
    nlong = a.split->nlong;
    nbuck = a.split->nbuck;
    nshort = a.split->nshort;
    nwork = nlong + nbuck + nshort;
  }
  uint32_t par = 0;  // work slot: the next pop writes the other one, so one barrier per pop
  // thread 0 pops each item one item ahead: the atomic's round trip runs while
  // the current item is sorted, and its value is stored only before the pop
  // barrier
  uint32_t next_w = 0;
  if (c.tid == 0) next_w = atomicAdd(&a.hdr->work_counter[0], 1u);
  while (true) {
    if (c.tid == 0) s_work[par] = next_w;
    __syncthreads();  // also: the previous item's shared buffers are free
    const int64_t w = s_work[par];
    par ^= 1u;
    if (w >= nwork) break;
    if (c.tid == 0) next_w = atomicAdd(&a.hdr->work_counter[0], 1u);
    if (w >= nlong && w < nlong + nbuck) {  // a bucket of a big segment: from the workspace copy into the keys
      const BucketItem it = a.buckets[w - nlong];
      const int64_t g = a.seg_base + it.lo;
      const int64_t len = it.len;
      U *sk = a.alt_k + g;
      V *sv = HAS_V ? a.alt_v + g : nullptr;
      if (len <= CAP) {
        c.sort_small(sk, sv, a.keys + g, HAS_V ? a.vals + g : nullptr, int(len), sk, sv);
      } else {  // keys too clustered for the split: back into place, then through global memory
        c.copy(a.keys + g, HAS_V ? a.vals + g : nullptr, sk, sv, len);
        __syncthreads();
        c.sort_large(a.keys + g, HAS_V ? a.vals + g : nullptr, sk, sv, len);
      }
      continue;
    }
    const int64_t s = !a.order ? w
                      : !a.split  ? a.order[w]
                      : w < nlong ? a.order[w]
                                  : a.order[a.nseg - nshort + (w - nlong - nbuck)];
    const int64_t lo = a.off ? clamp_off(a.off[s], a.n) : s * a.tile_len;
    const int64_t hi0 = a.off ? clamp_off(a.off[s + 1], a.n) : ((lo + a.tile_len) < a.n ? lo + a.tile_len : a.n);
    const int64_t hi = hi0 < lo ? lo : hi0;
    const int64_t len = hi - lo;
    if (len <= 1) continue;
    const int64_t g = a.seg_base + lo;
    if (len <= CAP) {
      c.sort_small(a.keys + g, HAS_V ? a.vals + g : nullptr, a.keys + g, HAS_V ? a.vals + g : nullptr, int(len),
                   a.alt_k + g, HAS_V ? a.alt_v + g : nullptr);
    } else {
      c.sort_large(a.keys + g, HAS_V ? a.vals + g : nullptr, a.alt_k + g, HAS_V ? a.alt_v + g : nullptr, len);
    }
  }
}

}  // namespace ak
