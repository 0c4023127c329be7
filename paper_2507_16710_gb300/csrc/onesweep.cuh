// onesweep.cuh -- LSD radix sort with one kernel per 8-bit digit.
//
// A sort of n keys of w bytes runs:
//   hist_kernel      one read of all keys; counts of every digit of every pass
//   plan_kernel      exclusive scan of each pass's 256 counts; marks "trivial"
//                    passes (one digit holds all n keys: a stable no-op) so they
//                    move no data
//   onesweep_pass    per active pass: CTAs take tile ids in increasing order,
//                    stage each tile in shared memory with a bulk copy issued
//                    ahead of use, rank keys by digit with a warp multisplit,
//                    publish per-digit counts, find their global offsets by
//                    decoupled look-back over predecessor tiles (the
//                    "opportunistic look-back" scan the paper's accumulate
//                    uses, Sec. II-B), and write the tile out in digit order
//                    from shared memory so each warp stores contiguous runs
//   finish_kernel    copy-back when an odd number of passes moved data, or the
//                    identity permutation when none did
//
// Every pass is stable, so the composition is the stable sort under the key
// transform of common.cuh.  All waits are bounded by a timeout that sets the
// status word instead of trapping.
#pragma once

#include "common.cuh"
#include "learned.cuh"

namespace ak {

constexpr uint32_t INACTIVE = 0xFFFFFFFFu;

struct RadixPlan {
  uint32_t m;                    // passes that move data
  uint32_t q[MAX_PASSES];        // active index of each pass, or INACTIVE
  uint32_t fmt[MAX_PASSES];      // packed sortperm of 8-byte keys: the data format of each pass (PassFormat)
  uint32_t pad[7];
  unsigned long long bin_off[MAX_PASSES][RADIX];  // exclusive digit offsets
};

enum SortMode : int { MODE_INPLACE = 0, MODE_PERM = 1 };

// What a sortperm pass of 8-byte keys reads and writes.  Once the passes of
// the low 32 key bits are done, the sort needs only the upper 32 bits of each
// radix key, and those and the 32-bit index fit one 8-byte word.  So the last
// active pass of the low half writes (upper radix-key half << 32 | index)
// words (PACK_OUT) and the passes of the upper half move those 8-byte words
// alone, keys only, and the last one writes the index (PACKED_IN): 16 instead
// of 24 bytes per key and pass.  PLAIN: key and index, as every other sort.
enum PassFormat : int { FMT_PLAIN = 0, FMT_PACK_OUT = 1, FMT_PACKED_IN = 2 };

// Look-back status word: 2 flag bits over a 30-bit (u32) or 62-bit (u64) count.
template <typename S> struct StatusWord;
template <> struct StatusWord<uint32_t> {
  static constexpr int SHIFT = 30;
  static constexpr uint32_t MASK = (1u << 30) - 1;
};
template <> struct StatusWord<unsigned long long> {
  static constexpr int SHIFT = 62;
  static constexpr unsigned long long MASK = (1ull << 62) - 1;
};
constexpr uint32_t FLAG_AGG = 1, FLAG_INC = 2;

template <typename U, typename V>
struct PassArgs {
  const U *k_in;      // source of the first active pass
  U *k_final;         // MODE_INPLACE: the caller's key buffer
  U *k_alt0, *k_alt1; // ping-pong buffers in the workspace
  const V *v_in;      // MODE_INPLACE pairs: caller values
  V *v_final;         // MODE_INPLACE: caller values; MODE_PERM: caller permutation
  V *v_alt;
  int64_t n;
  int pass;
  int kind;
  U flip;
  int mode;
  const RadixPlan *plan;
  void *status_cur;   // look-back words of this pass (zeroed)
  void *status_next;  // zeroed here for the next pass
  int64_t num_tiles;
  DevHeader *hdr;
  uint64_t timeout_ns;
  int debug_skip;     // AK_DEBUG_SKIP_FIRST_TILE: tile ids start at 1
  const LearnedModel *model;  // learned digits: bucket id of the key
  const uint32_t *gate;       // if set, run only when *gate == gate_want
  uint32_t gate_want;
  int64_t prefetch_ahead;     // one-tile CTAs: L2-prefetch the tile this many ids ahead (0: off)
  uint32_t *chunk_cnt;        // reduce-then-scan passes: digit counts of each chunk [chunk][RADIX]
  int64_t tiles_per_chunk;    // reduce-then-scan passes: consecutive tiles of one chunk (one CTA)
  int fmt_check;              // packed sortperm: run only when plan->fmt[pass] is this kernel's format
};

// Digit of a key in a pass: a radix digit, a byte of the learned bucket id
// evaluated from the key, or a byte of the value (a bucket id computed once and
// carried along as the value).
// DIGIT_GATHER (the low-memory sortperm): the index is the only data that
// moves; each pass reads a key through its index from the caller's keys.
enum DigitSource : int { DIGIT_RADIX = 0, DIGIT_LEARNED = 1, DIGIT_VALUE = 2, DIGIT_GATHER = 3 };

// ------------------------------------------------------------------ histogram
template <typename U, int BLOCK>
__global__ void __launch_bounds__(BLOCK) hist_kernel(const U *__restrict__ keys, int64_t n, int kind,
                                                     U flip, unsigned long long *counts,
                                                     uint4 *zero_buf, int64_t zero_vec,
                                                     const uint32_t *gate, uint32_t gate_want) {
  if (gate && *gate != gate_want) return;
  constexpr int PASSES = sizeof(U);
  __shared__ uint32_t sh[2][PASSES * RADIX];
  for (int i = threadIdx.x; i < 2 * PASSES * RADIX; i += BLOCK) (&sh[0][0])[i] = 0;
  const int64_t gtid = int64_t(blockIdx.x) * BLOCK + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * BLOCK;
  for (int64_t i = gtid; i < zero_vec; i += stride) zero_buf[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  uint32_t *h = sh[(threadIdx.x >> 5) & 1];
  auto count = [&](U u) {
    const U r = radix_key(u, kind, flip);
#pragma unroll
    for (int p = 0; p < PASSES; ++p) atomicAdd(&h[p * RADIX + digit_of(r, p * RADIX_BITS)], 1u);
  };
  constexpr int PER = 16 / sizeof(U);
  const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
  int64_t head = int64_t(((16 - (addr & 15)) & 15) / sizeof(U));
  if (head > n) head = n;
  for (int64_t i = gtid; i < head; i += stride) count(keys[i]);
  const int64_t nvec = (n - head) / PER;
  const uint4 *vk = reinterpret_cast<const uint4 *>(keys + head);
  for (int64_t i = gtid; i < nvec; i += stride) {
    uint4 x = __ldg(vk + i);
    const U *e = reinterpret_cast<const U *>(&x);
#pragma unroll
    for (int j = 0; j < PER; ++j) count(e[j]);
  }
  for (int64_t i = head + nvec * PER + gtid; i < n; i += stride) count(keys[i]);
  __syncthreads();
  for (int i = threadIdx.x; i < PASSES * RADIX; i += BLOCK) {
    const uint32_t c = sh[0][i] + sh[1][i];
    if (c) atomicAdd(&counts[i], (unsigned long long)c);
  }
}

// ----------------------------------------------------------------------- plan
// One CTA of RADIX threads.
static __global__ void __launch_bounds__(RADIX) plan_kernel(const unsigned long long *counts, int64_t n,
                                                     int passes, RadixPlan *plan, DevHeader *hdr,
                                                     int path_tag, const uint32_t *gate, uint32_t gate_want,
                                                     int pack_half = 0) {
  if (gate && *gate != gate_want) return;
  __shared__ unsigned long long scratch[RADIX / 32 + 1];
  __shared__ int triv[MAX_PASSES];
  if (threadIdx.x < MAX_PASSES) triv[threadIdx.x] = 0;
  __syncthreads();
  for (int p = 0; p < passes; ++p) {
    const unsigned long long c = counts[p * RADIX + threadIdx.x];
    if (c == (unsigned long long)n) triv[p] = 1;
    unsigned long long total;
    const unsigned long long ex = block_exclusive_scan<RADIX>(c, scratch, &total);
    plan->bin_off[p][threadIdx.x] = ex;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t m = 0;
    for (int p = 0; p < MAX_PASSES; ++p) plan->q[p] = (p < passes && !triv[p]) ? m++ : INACTIVE;
    plan->m = m;
    // packed sortperm (pack_half = passes of the low half): the last active
    // pass below pack_half packs, every active pass above it reads packed
    // words.  With no active low pass the first active upper pass packs,
    // unless it is the only one (then it writes the index directly).
    for (int p = 0; p < MAX_PASSES; ++p) plan->fmt[p] = FMT_PLAIN;
    if (pack_half > 0) {
      int low_last = -1, first_high = -1, last_active = -1;
      for (int p = 0; p < passes; ++p) {
        if (triv[p]) continue;
        last_active = p;
        if (p < pack_half) low_last = p;
        else if (first_high < 0) first_high = p;
      }
      if (first_high >= 0) {
        const int start = low_last >= 0 ? low_last : (first_high != last_active ? first_high : -1);
        if (start >= 0) {
          plan->fmt[start] = FMT_PACK_OUT;
          for (int p = start + 1; p < passes; ++p)
            if (!triv[p]) plan->fmt[p] = FMT_PACKED_IN;
        }
      }
    }
    hdr->info.radix_passes = int32_t(m);
    if (path_tag) hdr->info.path = path_tag;
  }
}

// ---------------------------------------------------------------- digit pass
// Digit of a key in a radix pass.  A 64-bit key's digit lies in one 32-bit
// half (a 128-bit key's in one 32-bit word, the same for every key of a pass),
// so only that word is transformed; the result equals digit_of(radix_key_t(k)).
template <int KIND, typename U>
__device__ __forceinline__ uint32_t radix_digit(U k, U flip, int shift) {
  if constexpr (sizeof(U) == 8) {
    const uint32_t lo = uint32_t(k), hi = uint32_t(uint64_t(k) >> 32);
    const bool upper = shift >= 32;
    uint32_t w = upper ? hi : lo;
    const uint32_t f = upper ? uint32_t(uint64_t(flip) >> 32) : uint32_t(flip);
    if constexpr (KIND == KIND_SINT) {
      if (upper) w ^= 0x80000000u;
    } else if constexpr (KIND == KIND_FLOAT) {
      const uint32_t neg = uint32_t(int32_t(hi) >> 31);  // negative: every bit flips
      w ^= neg | (upper ? 0x80000000u : 0u);             // otherwise only the sign bit
      const uint32_t mh = hi & 0x7FFFFFFFu;
      if (mh > 0x7FF00000u || (mh == 0x7FF00000u && lo != 0u)) w = 0xFFFFFFFFu;  // NaN: all ones
    }
    return ((w ^ f) >> (shift & 31)) & uint32_t(RADIX - 1);
  } else if constexpr (sizeof(U) == 16) {  // 128-bit integers: the 32-bit word of the digit
    const int wi = shift >> 5;
    uint32_t w = uint32_t(k >> (32 * wi)) ^ uint32_t(flip >> (32 * wi));
    if constexpr (KIND == KIND_SINT) {
      if (wi == 3) w ^= 0x80000000u;
    }
    return (w >> (shift & 31)) & uint32_t(RADIX - 1);
  } else {
    return digit_of(radix_key_t<KIND>(k, flip), shift);
  }
}

template <int DIGIT, int KIND, typename U, typename V>
__device__ __forceinline__ uint32_t pass_digit(const PassArgs<U, V> &a, U k, int shift) {
  if constexpr (DIGIT == DIGIT_LEARNED) return (lm_key_bucket<KIND>(a.model, k, a.flip) >> shift) & (RADIX - 1);
  else return radix_digit<KIND>(k, a.flip, shift);
}

// Shared memory of the digit pass: the staged tile (keys then values, filled
// by the bulk-copy engine), the same tile in digit order, and the ranking
// state.
template <typename U, typename V, bool HAS_V, int BLOCK, int ITEMS>
struct PassSmem {
  static constexpr int TILE = BLOCK * ITEMS;
  static constexpr int NW = BLOCK / 32;
  static constexpr int HROW = RADIX + 1;  // digit rows + the padding digit of a ragged tile
  static constexpr size_t KEYS = size_t(TILE) * sizeof(U);
  static constexpr size_t VALS = HAS_V ? size_t(TILE) * sizeof(V) : 0;
  static constexpr size_t STAGE = (KEYS + VALS + 127) / 128 * 128;
  static constexpr size_t OFF_OUT = STAGE;  // the tile in digit order
  // u16 warp counters, digit-major: row d holds the NW warps' counters of
  // digit d in NW/2 words plus one pad word, so consecutive rows start in
  // different banks
  static constexpr int HSTRIDE = NW / 2 + 1;  // 32-bit words per digit row (odd)
  static constexpr size_t OFF_HIST = OFF_OUT + STAGE;
  static constexpr size_t OFF_MASK = (OFF_HIST + size_t(HROW) * HSTRIDE * 4 + 15) / 16 * 16;  // u32[NW][HROW]
  static constexpr size_t OFF_DELTA = (OFF_MASK + size_t(NW) * HROW * 4 + 15) / 16 * 16;      // i32 or i64 [RADIX]
  static constexpr size_t OFF_SCR = OFF_DELTA + size_t(RADIX) * 8;                           // u32[RADIX/32]
  static constexpr size_t OFF_BAR = (OFF_SCR + (RADIX / 32) * 4 + 15) / 16 * 16;               // u64
  static constexpr size_t OFF_TILE = OFF_BAR + 8;                                            // i64: next tile
  static constexpr size_t OFF_FLAG = OFF_TILE + 8;                                           // u32
  static constexpr size_t OFF_DIG = (OFF_FLAG + 4 + 15) / 16 * 16;  // u8[TILE]: digit of each output slot
  static constexpr size_t BYTES = OFF_DIG + size_t(TILE);
  static_assert(TILE < 65536, "warp bases are u16");
  static_assert(NW % 2 == 0, "two 16-bit counters per word");
  static_assert(KEYS % 16 == 0 && STAGE % 128 == 0 && OFF_DELTA % 8 == 0 && OFF_BAR % 8 == 0 && OFF_TILE % 8 == 0,
                "shared-memory arrays aligned to their element size (bulk copies: 16 bytes)");
};

#ifndef AK_LOOKBACK_WINDOW
#define AK_LOOKBACK_WINDOW 8
#endif
constexpr int LOOKBACK_WINDOW = AK_LOOKBACK_WINDOW;  // predecessor words probed per round trip


// One digit pass.  Tile ids come from an atomic counter, so every predecessor
// of a tile is held by a CTA that already runs (forward progress of the
// look-back).  PERSIST: a wave of CTAs loops over tiles; a CTA claims its next
// tile as soon as the current tile's counts are published (a tile claimed
// earlier would hold up every later tile's look-back), pulls it into L2, and
// starts its bulk copy into the stage buffer once the current tile has left
// it, so the copy overlaps the look-back and the write-out.  Otherwise one CTA
// per tile, which also pulls the tile one residency wave ahead into L2.
//
// Per tile: (1) digit of every key, warp multisplit rank: peers of a digit
// found by OR-ing lane bits into a per-warp shared mask word, per-warp 16-bit
// counters, stable rank = running count + popc(peers below this lane);
// (2) per-digit tile counts published (flag AGG), a CTA scan of the 256 counts
// gives digit starts and warp bases; (3) scatter into the output buffer in
// digit order; (4) decoupled look-back, inclusive counts published (flag INC);
// (5) write-out: consecutive threads store consecutive slots of a digit run.
//
// RTS (reduce-then-scan, after chunk_hist_kernel): CTA c sorts the tiles of
// chunk c in increasing order; its digit offsets are the counts of chunks
// 0..c-1 plus, tile after tile, the counts of its own earlier tiles, held in a
// register of the digit's thread.  Nothing is published and no CTA waits on
// another.
// CTAs per SM the register budget is sized for (2 x 512, 3 x 384 threads).
constexpr int pass_min_blocks(int block) { return block >= 512 ? 2 : (block >= 384 ? 3 : 4); }

template <typename U, typename V, bool HAS_V, int KIND, typename S, int BLOCK, int ITEMS, bool PERSIST,
          int DIGIT = DIGIT_RADIX, bool RTS = false, int FMT = FMT_PLAIN>
__global__ void __launch_bounds__(BLOCK, pass_min_blocks(BLOCK)) onesweep_pass(PassArgs<U, V> a) {
  using L = PassSmem<U, V, HAS_V, BLOCK, ITEMS>;
  constexpr int TILE = L::TILE;
  constexpr int NW = L::NW;
  constexpr int HROW = L::HROW;
  constexpr int H2 = 2 * L::HSTRIDE;  // u16 slots per digit row
  static_assert(BLOCK >= RADIX, "one digit per thread in the scan and look-back");
  static_assert(DIGIT != DIGIT_VALUE || HAS_V, "a value-carried digit needs the value stream");
  static_assert(DIGIT != DIGIT_GATHER || HAS_V, "gathered keys need the index stream");
  static_assert(!RTS || (PERSIST && DIGIT == DIGIT_RADIX), "reduce-then-scan: persistent radix passes");
  static_assert(FMT == FMT_PLAIN || (sizeof(U) == 8 && std::is_same<V, uint32_t>::value && !RTS &&
                                     DIGIT == DIGIT_RADIX && HAS_V == (FMT == FMT_PACK_OUT)),
                "packed sortperm: 8-byte keys, u32 indices");
  constexpr bool GATHER = DIGIT == DIGIT_GATHER;  // keys are read through the index, never moved
  extern __shared__ __align__(128) uint8_t smem[];
  U *sk = reinterpret_cast<U *>(smem);
  V *sv = reinterpret_cast<V *>(smem + L::KEYS);
  U *ok = reinterpret_cast<U *>(smem + L::OFF_OUT);
  V *ov = reinterpret_cast<V *>(smem + L::OFF_OUT + L::KEYS);
  uint16_t *whist = reinterpret_cast<uint16_t *>(smem + L::OFF_HIST);
  uint32_t *whist32 = reinterpret_cast<uint32_t *>(smem + L::OFF_HIST);
  uint32_t *wmask = reinterpret_cast<uint32_t *>(smem + L::OFF_MASK);
  // per digit: destination index of output slot 0 (32-bit when every index fits)
  using Delta = typename std::conditional<sizeof(S) == 4, int32_t, long long>::type;
  Delta *s_delta = reinterpret_cast<Delta *>(smem + L::OFF_DELTA);
  uint32_t *s_scr = reinterpret_cast<uint32_t *>(smem + L::OFF_SCR);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::OFF_BAR);
  long long *s_next = reinterpret_cast<long long *>(smem + L::OFF_TILE);
  uint32_t *s_flag = reinterpret_cast<uint32_t *>(smem + L::OFF_FLAG);
  uint8_t *s_dig = smem + L::OFF_DIG;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (a.gate && *a.gate != a.gate_want) return;
  // packed sortperm: the variants of a pass are all launched; the plan's one runs
  if (a.fmt_check && a.plan->fmt[a.pass] != uint32_t(FMT)) return;

  // Clear the next pass's look-back rows (the grid covers rows blockIdx.x + k*gridDim.x).
  if (a.status_next) {
    S *nx = reinterpret_cast<S *>(a.status_next);
    for (int64_t r = blockIdx.x; r < a.num_tiles; r += gridDim.x)
      for (int i = tid; i < RADIX; i += BLOCK) nx[r * RADIX + i] = S(0);
  }
  const uint32_t q = a.plan->q[a.pass];
  if (q == INACTIVE) return;
  const uint32_t m = a.plan->m;

  // source / destination of this active pass
  const U *ksrc;
  U *kdst;
  const V *vsrc = nullptr;
  V *vdst = nullptr;
  bool write_keys = true, gen_index = false;
  if (a.mode == MODE_INPLACE) {
    kdst = (q & 1) ? a.k_final : a.k_alt0;
    ksrc = (q == 0) ? a.k_in : ((q & 1) ? a.k_alt0 : a.k_final);
    if (HAS_V) {
      vdst = (q & 1) ? a.v_final : a.v_alt;
      vsrc = (q == 0) ? a.v_in : ((q & 1) ? a.v_alt : a.v_final);
    }
  } else {
    kdst = (q & 1) ? a.k_alt1 : a.k_alt0;
    ksrc = (q == 0) ? a.k_in : ((q & 1) ? a.k_alt0 : a.k_alt1);
    write_keys = (q + 1 != m);
    auto vbuf = [&](uint32_t qq) { return (((m - 1 - qq) & 1) == 0) ? a.v_final : a.v_alt; };
    vdst = vbuf(q);
    if (q == 0) gen_index = true;
    else vsrc = vbuf(q - 1);
  }
  const bool load_v = HAS_V && !gen_index;
  const bool load_k = !GATHER;  // the stage holds the tile's keys (gathered keys are read in the ranking)
  if (GATHER) write_keys = false;
  const bool aligned = (!load_k || ((reinterpret_cast<uintptr_t>(ksrc) & 15) == 0)) &&
                       (!load_v || ((reinterpret_cast<uintptr_t>(vsrc) & 15) == 0));
  const int64_t full_tiles = a.n / TILE;  // tiles that need no bounds checks
  auto is_bulk = [&](int64_t t) { return aligned && t < full_tiles && (load_k || load_v); };
  uint32_t phase = 0;     // thread 0: parity of the next completion of bar
  bool pending = false;   // thread 0: a bulk copy is in flight
  auto claim = [&]() -> int64_t {
    const int64_t t = int64_t(atomicAdd(&a.hdr->tile_counter[a.pass], 1u)) + (a.debug_skip ? 1 : 0);
    return t < a.num_tiles ? t : a.num_tiles;
  };
  constexpr int CLAIMER = BLOCK - 1;  // claims the next tile; not a look-back thread when BLOCK > RADIX
  auto issue = [&](int64_t t) {  // thread 0 only; the stage buffer must be free
    if (t < a.num_tiles && is_bulk(t)) {
      mbar_expect_tx(bar, uint32_t((load_k ? L::KEYS : 0) + (load_v ? L::VALS : 0)));
      if (load_k) bulk_g2s(sk, ksrc + t * TILE, uint32_t(L::KEYS), bar);
      if (load_v) bulk_g2s(sv, vsrc + t * TILE, uint32_t(L::VALS), bar);
      pending = true;
    }
  };
  auto prefetch_l2 = [&](int64_t t) {  // thread 0 only
    if (t < full_tiles && aligned) {
      if (load_k) bulk_prefetch_l2(ksrc + t * TILE, uint32_t(L::KEYS));
      if (load_v) bulk_prefetch_l2(vsrc + t * TILE, uint32_t(L::VALS));
    }
  };

  for (int i = tid; i < NW * HROW; i += BLOCK) wmask[i] = 0u;
  for (int i = tid; i < HROW * L::HSTRIDE; i += BLOCK) whist32[i] = 0u;
  int64_t next_tile = 0;  // CLAIMER: the tile claimed for the next iteration
  // RTS: this CTA's chunk of tiles [rts_first, rts_end)
  const int64_t rts_first = RTS ? (int64_t(blockIdx.x) * a.tiles_per_chunk < a.num_tiles
                                       ? int64_t(blockIdx.x) * a.tiles_per_chunk : a.num_tiles)
                                : 0;
  const int64_t rts_end = RTS ? (rts_first + a.tiles_per_chunk < a.num_tiles ? rts_first + a.tiles_per_chunk
                                                                              : a.num_tiles)
                              : 0;
  if (tid == 0) {
    mbar_init(bar, 1);
    const int64_t t = RTS ? rts_first : claim();
    *s_next = (long long)t;
    issue(t);
    // one-tile CTAs: pull the tile about one residency wave ahead into L2 so
    // HBM stays busy while CTAs rank, look back and write
    if (!PERSIST && a.prefetch_ahead > 0) prefetch_l2(t + a.prefetch_ahead);
    *s_flag = 0;
  }
  __syncthreads();

  const int shift = a.pass * RADIX_BITS;
  // FMT_PACK_OUT: the upper half of the radix key over the index
  auto pack_word = [&](U k, V idx) -> U {
    if constexpr (sizeof(U) == 8) return U((uint64_t(radix_key_t<KIND>(k, a.flip)) & 0xFFFFFFFF00000000ull) | uint64_t(idx));
    else return k;
  };
  const uint32_t lt_mask = lanemask_lt();
  const uint32_t gt_mask = ~(lt_mask | (1u << lane));
  uint32_t *wm = wmask + warp * HROW;
  S *st = reinterpret_cast<S *>(a.status_cur);
  // RTS: keys of digit tid in chunks before this one, then in this chunk's
  // tiles so far (independent loads, 32 in flight per round)
  unsigned long long run = 0;
  if constexpr (RTS) {
    if (tid < RADIX) {
      constexpr int UNR = 32;
      const int64_t nc = blockIdx.x;
      for (int64_t c0 = 0; c0 < nc; c0 += UNR) {
        uint32_t v[UNR];
#pragma unroll
        for (int j = 0; j < UNR; ++j) v[j] = (c0 + j < nc) ? a.chunk_cnt[(c0 + j) * RADIX + tid] : 0u;
#pragma unroll
        for (int j = 0; j < UNR; ++j) run += v[j];
      }
    }
  }

  for (;;) {
    const int64_t tile = *s_next;  // written by thread 0 before barriers B and C of the previous tile
    if (tile >= a.num_tiles) break;
    if (tid == 0 && pending) {
      if (mbar_wait_bounded(bar, phase, a.timeout_ns)) {
        pending = false;
        phase ^= 1u;
      } else {  // the copy is still owed: the exit path waits for it again
        set_error(a.hdr, AK_ERR_TIMEOUT);
        *s_flag = 1;
      }
    }
    __syncthreads();  // S: the tile is resident; the previous tile is fully written out
    if (*s_flag) break;

    const int64_t base = tile * TILE;
    const int tile_n = int((a.n - base) < int64_t(TILE) ? (a.n - base) : int64_t(TILE));
    if (!is_bulk(tile)) {  // ragged last tile or unaligned source: plain loads
      if (load_k)
        for (int i = tid; i < tile_n; i += BLOCK) sk[i] = ksrc[base + i];
      if (load_v)
        for (int i = tid; i < tile_n; i += BLOCK) sv[i] = vsrc[base + i];
      __syncthreads();
    }

    auto body = [&](auto full_tag) {
      constexpr bool FULL = decltype(full_tag)::value;
      // ---- warp multisplit ranking (item i of lane l sits at wbase + 32 i + l)
      const int wbase = warp * 32 * ITEMS;
      uint32_t dr[ITEMS];  // rank << 9 | digit (digit RADIX marks a padding slot)
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int idx = wbase + i * 32 + lane;
        if constexpr (DIGIT == DIGIT_VALUE)
          dr[i] = (FULL || idx < tile_n) ? ((uint32_t(sv[idx]) >> shift) & uint32_t(RADIX - 1)) : uint32_t(RADIX);
        else if constexpr (GATHER)  // the key of this item's index, from the caller's keys
          dr[i] = (FULL || idx < tile_n)
                      ? pass_digit<DIGIT_RADIX, KIND>(a, a.k_in[gen_index ? base + idx : int64_t(sv[idx])], shift)
                      : uint32_t(RADIX);
        else
          dr[i] = (FULL || idx < tile_n) ? pass_digit<DIGIT, KIND>(a, sk[idx], shift) : uint32_t(RADIX);
      }
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const uint32_t d = dr[i];
        uint16_t *wc = whist + d * H2 + warp;  // this warp's running count of digit d
        atomicOr(&wm[d], 1u << lane);
        __syncwarp();
        const uint32_t peers = wm[d];
        const uint32_t cnt = *wc;
        __syncwarp();
        if ((peers & gt_mask) == 0) {  // highest lane of the group updates and resets
          *wc = uint16_t(cnt + __popc(peers));
          wm[d] = 0u;
        }
        __syncwarp();
        dr[i] = ((cnt + __popc(peers & lt_mask)) << 9) | d;
      }
      __syncthreads();  // A: every warp row complete

      // ---- tile counts, publish, digit scan
      uint32_t my_cnt = 0, inc = 0;
      uint32_t *hrow = whist32 + tid * L::HSTRIDE;
      if (tid < RADIX) {
#pragma unroll
        for (int v = 0; v < NW / 2; ++v) {
          const uint32_t w = hrow[v];
          my_cnt += (w & 0xFFFFu) + (w >> 16);
        }
        if constexpr (!RTS)
          st_relaxed(&st[tile * RADIX + tid], (S(tile == 0 ? FLAG_INC : FLAG_AGG) << StatusWord<S>::SHIFT) | S(my_cnt));
        inc = warp_inclusive_scan(my_cnt);
        if (lane == 31) s_scr[warp] = inc;
      }

      __syncthreads();  // A2: warp totals of the digit scan; this tile's counts are published
      // the next tile is claimed only now (a claimed tile whose counts are not
      // yet published would hold up every later tile's look-back); the claim's
      // round trip overlaps the scan and scatter
      if (PERSIST && tid == CLAIMER) {
        if constexpr (RTS) next_tile = tile + 1 < rts_end ? tile + 1 : a.num_tiles;
        else next_tile = claim();
      }
      uint32_t start = 0;
      if (tid < RADIX) {
        start = inc - my_cnt;
#pragma unroll
        for (int w2 = 0; w2 < RADIX / 32; ++w2)
          if (w2 < warp) start += s_scr[w2];
        uint32_t run = start;  // warp bases: digit start + counts of earlier warps
#pragma unroll
        for (int v = 0; v < NW / 2; ++v) {
          const uint32_t w = hrow[v];
          const uint32_t lo = run, hi = run + (w & 0xFFFFu);
          run = hi + (w >> 16);
          hrow[v] = (lo & 0xFFFFu) | (hi << 16);
        }
      }

      // ---- scatter into the output buffer in digit order (this thread's items)
      auto scatter = [&]() {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
          const uint32_t d = dr[i] & 511u;
          if (FULL || d < RADIX) {
            const int idx = wbase + i * 32 + lane;
            const uint32_t pos = uint32_t(whist[d * H2 + warp]) + (dr[i] >> 9);
            if (!GATHER) ok[pos] = sk[idx];
            if (HAS_V) ov[pos] = gen_index ? V(base + idx) : sv[idx];
            s_dig[pos] = uint8_t(d);
          }
        }
      };
      // ---- decoupled look-back of digit d (count cnt) over a window of
      // predecessors per probe; publishes the inclusive count, returns the
      // exclusive prefix
      auto lookback = [&](int d, uint32_t cnt) -> unsigned long long {
        unsigned long long excl = 0;
        if (tile > 0) {
          int64_t j = tile - 1;
          uint64_t t0 = 0;
          uint32_t spins = 0;
          for (;;) {
            S lb[LOOKBACK_WINDOW];  // lb[k]: status word of predecessor j - k
#pragma unroll
            for (int k = 0; k < LOOKBACK_WINDOW; ++k) lb[k] = (j - k >= 0) ? ld_relaxed(&st[(j - k) * RADIX + d]) : S(0);
            int used = 0;
            bool done = false, stop = false;
#pragma unroll
            for (int k = 0; k < LOOKBACK_WINDOW; ++k) {
              const uint32_t flag = uint32_t(lb[k] >> StatusWord<S>::SHIFT);
              if (!stop) {
                if (flag == 0) {
                  stop = true;  // not published yet (tile 0 publishes INC, so j - k >= 0 here)
                } else {
                  excl += (unsigned long long)(lb[k] & StatusWord<S>::MASK);
                  ++used;
                  if (flag == FLAG_INC) done = stop = true;
                }
              }
            }
            if (done) break;
            j -= used;
            if (used == 0) {
              __nanosleep(64);  // predecessor not published yet: yield issue slots
              if ((++spins & 31u) == 0) {
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > a.timeout_ns) {
                  // partial sums of published predecessors keep every store in bounds
                  set_error(a.hdr, AK_ERR_TIMEOUT);
                  break;
                }
              }
            }
          }
          st_relaxed(&st[tile * RADIX + d], (S(FLAG_INC) << StatusWord<S>::SHIFT) | S(excl + cnt));
        }
        return excl;
      };

      __syncthreads();  // B: warp bases ready
      scatter();
      if (tid < RADIX) {
        unsigned long long excl;
        if constexpr (RTS) {
          excl = run;
          run += my_cnt;
        } else {
          excl = lookback(tid, my_cnt);
        }
        s_delta[tid] = Delta((long long)(a.plan->bin_off[a.pass][tid] + excl) - (long long)start);
      }
      if (PERSIST && tid == CLAIMER) {
        *s_next = (long long)next_tile;
        prefetch_l2(next_tile);
      }

      __syncthreads();  // C: output buffer and destinations ready; the stage buffer is free
      if (PERSIST) {
        if (tid == 0) issue(*s_next);  // lands while this tile is written out
        // counters of the next tile (barrier S separates this from its ranking)
        for (int i = tid; i < HROW * L::HSTRIDE; i += BLOCK) whist32[i] = 0u;
      }

      // ---- write the tile out: consecutive threads store consecutive slots of a digit run
      if (FULL) {
        constexpr int WB = ITEMS % 4 == 0 ? 4 : (ITEMS % 3 == 0 ? 3 : (ITEMS % 2 == 0 ? 2 : 1));
#pragma unroll
        for (int r0 = 0; r0 < ITEMS; r0 += WB) {  // WB slots per thread: all loads before the stores
          U k[WB];
          long long dst[WB];
#pragma unroll
          for (int r = 0; r < WB; ++r) {
            const int i = (r0 + r) * BLOCK + tid;
            k[r] = GATHER ? U(0) : ok[i];
            dst[r] = (long long)s_delta[s_dig[i]] + i;
          }
#pragma unroll
          for (int r = 0; r < WB; ++r) {
            if constexpr (FMT == FMT_PACK_OUT) {
              kdst[dst[r]] = pack_word(k[r], ov[(r0 + r) * BLOCK + tid]);
            } else {
              if (write_keys) kdst[dst[r]] = k[r];
              else if constexpr (FMT == FMT_PACKED_IN) a.v_final[dst[r]] = V(k[r]);  // the index half
              if (HAS_V) vdst[dst[r]] = ov[(r0 + r) * BLOCK + tid];
            }
          }
        }
      } else {
        for (int i = tid; i < tile_n; i += BLOCK) {
          const U k = GATHER ? U(0) : ok[i];
          const long long dst = (long long)s_delta[s_dig[i]] + i;
          if constexpr (FMT == FMT_PACK_OUT) {
            kdst[dst] = pack_word(k, ov[i]);
          } else {
            if (write_keys) kdst[dst] = k;
            else if constexpr (FMT == FMT_PACKED_IN) a.v_final[dst] = V(k);
            if (HAS_V) vdst[dst] = ov[i];
          }
        }
      }
    };
    if (tile_n == TILE) body(std::true_type{});
    else body(std::false_type{});

    if (!PERSIST) break;  // one tile per CTA
  }
  // a copy left in flight by a timed-out wait must land before the CTA exits
  if (tid == 0 && pending) mbar_wait_bounded(bar, phase, a.timeout_ns);
}

// --------------------------------------------------- reduce-then-scan upsweep
// Digit counts of one pass over one chunk (tiles_per_chunk consecutive tiles,
// the range one CTA of the following reduce-then-scan pass sorts in order).
// The pass then needs no look-back: chunk c's keys of digit d start after the
// keys of smaller digits (the plan's bin offsets) and after chunks 0..c-1's
// keys of digit d, and inside the chunk its CTA keeps a running count per
// digit from tile to tile.
template <typename U, typename V, int KIND, int BLOCK>
__global__ void __launch_bounds__(BLOCK) chunk_hist_kernel(PassArgs<U, V> a, int tile_keys) {
  if (a.gate && *a.gate != a.gate_want) return;
  const uint32_t q = a.plan->q[a.pass];
  if (q == INACTIVE) return;
  // the keys this active pass reads (the pass's own choice of source buffer)
  const U *ksrc = (q == 0) ? a.k_in : ((q & 1) ? a.k_alt0 : (a.mode == MODE_INPLACE ? a.k_final : a.k_alt1));
  constexpr int NSUB = BLOCK / 64;  // one sub-histogram per pair of warps
  __shared__ uint32_t h[NSUB][RADIX];
  for (int i = threadIdx.x; i < NSUB * RADIX; i += BLOCK) (&h[0][0])[i] = 0u;
  __syncthreads();
  const int64_t b = int64_t(blockIdx.x) * a.tiles_per_chunk * tile_keys;
  int64_t e = b + a.tiles_per_chunk * tile_keys;
  if (e > a.n) e = a.n;
  uint32_t *hh = h[threadIdx.x >> 6];
  const int shift = a.pass * RADIX_BITS;
  auto count = [&](U k) { atomicAdd(&hh[radix_digit<KIND>(k, a.flip, shift)], 1u); };
  if (b < e && (reinterpret_cast<uintptr_t>(ksrc + b) & 15) == 0) {
    constexpr int PER = 16 / sizeof(U);
    constexpr int UNR = 4;  // 64 bytes in flight per thread
    const int64_t nvec = (e - b) / PER;
    const uint4 *vk = reinterpret_cast<const uint4 *>(ksrc + b);
    int64_t i = threadIdx.x;
    for (; i + (UNR - 1) * BLOCK < nvec; i += UNR * BLOCK) {
      uint4 x[UNR];
#pragma unroll
      for (int j = 0; j < UNR; ++j) x[j] = __ldg(vk + i + j * BLOCK);
#pragma unroll
      for (int j = 0; j < UNR; ++j) {
        const U *el = reinterpret_cast<const U *>(&x[j]);
#pragma unroll
        for (int t = 0; t < PER; ++t) count(el[t]);
      }
    }
    for (; i < nvec; i += BLOCK) {
      const uint4 x = __ldg(vk + i);
      const U *el = reinterpret_cast<const U *>(&x);
#pragma unroll
      for (int t = 0; t < PER; ++t) count(el[t]);
    }
    for (int64_t k = b + nvec * PER + threadIdx.x; k < e; k += BLOCK) count(ksrc[k]);
  } else {
    for (int64_t k = b + threadIdx.x; k < e; k += BLOCK) count(ksrc[k]);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RADIX; d += BLOCK) {
    uint32_t c = 0;
#pragma unroll
    for (int s2 = 0; s2 < NSUB; ++s2) c += h[s2][d];
    a.chunk_cnt[int64_t(blockIdx.x) * RADIX + d] = c;
  }
}

// --------------------------------------------------------------------- finish
template <typename U, typename V, bool HAS_V>
__global__ void finish_kernel(PassArgs<U, V> a) {
  if (a.gate && *a.gate != a.gate_want) return;
  const uint32_t m = a.plan->m;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (a.mode == MODE_INPLACE) {
    if ((m & 1u) == 0) return;  // the last active pass wrote the caller's buffers
    for (int64_t i = t; i < a.n; i += stride) {
      a.k_final[i] = a.k_alt0[i];
      if (HAS_V) a.v_final[i] = a.v_alt[i];
    }
  } else {
    if (m != 0) return;
    for (int64_t i = t; i < a.n; i += stride) a.v_final[i] = V(i);  // all keys tie
  }
}

}  // namespace ak
