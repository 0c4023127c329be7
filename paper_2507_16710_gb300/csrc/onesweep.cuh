// onesweep.cuh -- LSD radix sort with one kernel per 8-bit digit.
//
// A sort of n keys of w bytes runs:
//   hist_kernel      one read of all keys; counts of every digit of every pass
//   plan_kernel      exclusive scan of each pass's 256 counts; marks "trivial"
//                    passes (one digit holds all n keys: a stable no-op) so they
//                    move no data
//   onesweep_pass    per active pass: each CTA takes the next tile id, stages
//                    the tile in shared memory with one bulk copy, ranks keys by
//                    digit with a warp multisplit (match.any), publishes its
//                    per-digit counts, finds its global offsets by decoupled
//                    look-back over predecessor tiles (the "opportunistic
//                    look-back" scan the paper's accumulate uses, Sec. II-B), and
//                    writes the tile out in digit order from shared memory so
//                    each warp stores contiguous runs
//   finish_kernel    copy-back when an odd number of passes moved data, or the
//                    identity permutation when none did
//
// Every pass is stable, so the composition is the stable sort under the key
// transform of common.cuh.  All waits are bounded by a timeout that sets the
// status word instead of trapping.
#pragma once

#include "common.cuh"
#include "learned.cuh"

// Warp matcher used by the digit passes (see warp_peers below).
#ifndef AK_WARP_MATCH
#define AK_WARP_MATCH 2
#endif

namespace ak {

constexpr uint32_t INACTIVE = 0xFFFFFFFFu;

struct RadixPlan {
  uint32_t m;                    // passes that move data
  uint32_t q[MAX_PASSES];        // active index of each pass, or INACTIVE
  uint32_t pad[7];
  unsigned long long bin_off[MAX_PASSES][RADIX];  // exclusive digit offsets
};

enum SortMode : int { MODE_INPLACE = 0, MODE_PERM = 1 };

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
};

// Digit of a key in a pass: a radix digit, or a byte of the learned bucket id.
enum DigitSource : int { DIGIT_RADIX = 0, DIGIT_LEARNED = 1 };
template <int DIGIT, int KIND, typename U, typename V>
__device__ __forceinline__ uint32_t pass_digit(const PassArgs<U, V> &a, U k, int shift) {
  if constexpr (DIGIT == DIGIT_LEARNED) return (lm_key_bucket<KIND>(a.model, k, a.flip) >> shift) & (RADIX - 1);
  else return digit_of(radix_key_t<KIND>(k, a.flip), shift);
}

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
                                                     int path_tag, const uint32_t *gate, uint32_t gate_want) {
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
    hdr->info.radix_passes = int32_t(m);
    if (path_tag) hdr->info.path = path_tag;
  }
}

// ---------------------------------------------------------------- digit pass
// Persistent CTAs walk tiles in increasing id order (ids from an atomic counter).
// A ring of STAGES shared-memory tile buffers is filled by the bulk-copy engine
// ahead of use, so loads of later tiles overlap the ranking, look-back and
// write-out of the current one.  Forward progress of the look-back: every CTA
// processes the tiles it holds in increasing order, so the holder of the
// smallest unfinished tile only waits on finished tiles.
template <typename U, typename V, bool HAS_V, int BLOCK, int ITEMS, int STAGES, int DIGIT = DIGIT_RADIX>
struct PassSmem {
  static constexpr int TILE = BLOCK * ITEMS;
  static constexpr int NW = BLOCK / 32;
  static constexpr int HROW = RADIX + 2;  // u16 per warp row: digits + the invalid-key slot
  static constexpr size_t KEYS = size_t(TILE) * sizeof(U);
  static constexpr size_t VALS = HAS_V ? size_t(TILE) * sizeof(V) : 0;
  static constexpr size_t STAGE = (KEYS + VALS + 127) / 128 * 128;
  static constexpr size_t OFF_OUT = STAGE * STAGES;  // the tile in digit order
  static constexpr size_t OFF_HIST = OFF_OUT + STAGE;
  // OFF_HIST: u16 counters, digit-major: row d holds the NW warps' counters of
  // digit d in NW/2 words plus one pad word, so rows start in distinct banks
  static constexpr int HSTRIDE = NW / 2 + 1;  // 32-bit words per digit row (odd)
  static constexpr size_t OFF_MASK = (OFF_HIST + size_t(HROW) * HSTRIDE * 4 + 15) / 16 * 16;  // u32[NW][HROW]
  static constexpr size_t MASK_BYTES = AK_WARP_MATCH == 3 ? 8 : 4;                          // per digit and warp
  static constexpr size_t OFF_KPTR = OFF_MASK + size_t(NW) * HROW * MASK_BYTES;             // u64[RADIX]
  static constexpr size_t OFF_VPTR = OFF_KPTR + RADIX * 8;                                  // u64[RADIX]
  static constexpr size_t OFF_SCR = OFF_VPTR + (HAS_V ? RADIX * 8 : 0);                     // u32[NW+1]
  static constexpr size_t OFF_BAR = (OFF_SCR + (NW + 1) * 4 + 15) / 16 * 16;             // u64[STAGES]
  static constexpr size_t OFF_TILE = OFF_BAR + 8 * STAGES;                                // u32[STAGES]
  static constexpr size_t OFF_FLAG = OFF_TILE + 4 * STAGES;                               // u32
  static constexpr size_t OFF_DIG = OFF_FLAG + 16;  // u8[TILE]: digits in tile order (learned digits)
  static constexpr size_t BYTES = OFF_DIG + (DIGIT == DIGIT_LEARNED ? size_t(TILE) : 0);
  static_assert(TILE < 65536, "warp bases are u16");
  static_assert(NW % 2 == 0, "two 16-bit counters per word");
  static_assert(KEYS % 16 == 0 && STAGE % 128 == 0 && OFF_MASK % 16 == 0 && OFF_KPTR % 8 == 0 &&
                    OFF_BAR % 8 == 0,
                "shared-memory arrays aligned to their element size (bulk copies: 16 bytes)");
};

constexpr int LOOKBACK_WINDOW = 8;  // predecessor words probed per round trip

// Lanes of the warp holding the same digit.  AK_WARP_MATCH selects match.any
// (0), a bit-sliced match from ballots (1: the peers of a lane are the lanes
// agreeing on every bit; 9 bits when the padding digit RADIX can occur), a
// shared-memory mask per digit that every lane ORs its bit into (2, default:
// fixed cost), or the same with two items per step in 64-bit masks (3: half the
// dependent round trips but twice the mask memory; measured slower on GB300).
// (AK_WARP_MATCH is defined at the top of this file.)
__device__ __forceinline__ uint32_t warp_peers(uint32_t d, bool nine_bits) {
#if AK_WARP_MATCH == 0
  (void)nine_bits;
  return __match_any_sync(0xffffffffu, d);
#else
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
    peers &= ((d >> b) & 1u) ? bal : ~bal;
  }
  if (nine_bits) {
    const uint32_t bal = __ballot_sync(0xffffffffu, (d >> 8) & 1u);
    peers &= ((d >> 8) & 1u) ? bal : ~bal;
  }
  return peers;
#endif
}

template <typename U, typename V, bool HAS_V, int KIND, typename S, int BLOCK, int ITEMS, int STAGES,
          bool PERSIST, int DIGIT = DIGIT_RADIX>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) onesweep_pass(PassArgs<U, V> a) {
  using L = PassSmem<U, V, HAS_V, BLOCK, ITEMS, STAGES, DIGIT>;
  constexpr int TILE = L::TILE;
  constexpr int NW = L::NW;
  constexpr int HROW = L::HROW;
  static_assert(BLOCK >= RADIX, "one digit per thread in the look-back");
  static_assert(PERSIST ? STAGES >= 2 : STAGES == 1, "stage ring");
  extern __shared__ __align__(128) uint8_t smem[];
  uint16_t *whist = reinterpret_cast<uint16_t *>(smem + L::OFF_HIST);
  uint32_t *wmask = reinterpret_cast<uint32_t *>(smem + L::OFF_MASK);
  unsigned long long *wmask2 = reinterpret_cast<unsigned long long *>(smem + L::OFF_MASK);
  // per digit: address of the destination of tile position 0 (base + delta,
  // kept as an integer; base + delta + i is inside the buffer for every key)
  unsigned long long *s_kptr = reinterpret_cast<unsigned long long *>(smem + L::OFF_KPTR);
  unsigned long long *s_vptr = reinterpret_cast<unsigned long long *>(smem + L::OFF_VPTR);
  uint32_t *s_scr = reinterpret_cast<uint32_t *>(smem + L::OFF_SCR);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::OFF_BAR);
  uint32_t *s_tile = reinterpret_cast<uint32_t *>(smem + L::OFF_TILE);
  uint32_t *s_flag = reinterpret_cast<uint32_t *>(smem + L::OFF_FLAG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *s_dig = smem + L::OFF_DIG;
  if (a.gate && *a.gate != a.gate_want) return;

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
  const bool aligned = ((reinterpret_cast<uintptr_t>(ksrc) & 15) == 0) &&
                       (!load_v || ((reinterpret_cast<uintptr_t>(vsrc) & 15) == 0));
  const int64_t full_tiles = a.n / TILE;  // tiles that need no bounds checks
  auto is_bulk = [&](int64_t t) { return aligned && t < full_tiles; };
  const uint32_t tx_bytes = uint32_t(L::KEYS + (load_v ? L::VALS : 0));
  auto stage_keys = [&](int s) { return reinterpret_cast<U *>(smem + size_t(s) * L::STAGE); };
  auto stage_vals = [&](int s) { return reinterpret_cast<V *>(smem + size_t(s) * L::STAGE + L::KEYS); };
  auto next_tile = [&]() -> int64_t {
    return int64_t(atomicAdd(&a.hdr->tile_counter[a.pass], 1u)) + (a.debug_skip ? 1 : 0);
  };
  auto issue = [&](int s, int64_t t) {  // thread 0 only
    if (t < a.num_tiles && is_bulk(t)) {
      mbar_expect_tx(&bar[s], tx_bytes);
      bulk_g2s(stage_keys(s), ksrc + t * TILE, uint32_t(L::KEYS), &bar[s]);
      if (load_v) bulk_g2s(stage_vals(s), vsrc + t * TILE, uint32_t(L::VALS), &bar[s]);
    }
  };

  for (int i = tid; i < NW * HROW * int(L::MASK_BYTES / 4); i += BLOCK) wmask[i] = 0u;
  for (int i = tid; i < HROW * L::HSTRIDE; i += BLOCK) reinterpret_cast<uint32_t *>(whist)[i] = 0u;
  uint32_t phase_bits = 0;  // thread 0: parity to wait for, per stage
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    for (int s = 0; s < STAGES; ++s) {
      const int64_t t = next_tile();
      s_tile[s] = uint32_t(t < a.num_tiles ? t : a.num_tiles);
      issue(s, t);
      // one-tile CTAs: pull the tile about one residency wave ahead into L2 so
      // HBM stays busy while CTAs rank, look back and write
      if (!PERSIST && a.prefetch_ahead > 0) {
        const int64_t tp = t + a.prefetch_ahead;
        if (tp < full_tiles && aligned) {
          bulk_prefetch_l2(ksrc + tp * TILE, uint32_t(L::KEYS));
          if (load_v) bulk_prefetch_l2(vsrc + tp * TILE, uint32_t(L::VALS));
        }
      }
    }
    *s_flag = 0;
    // the first stage must be resident before the loop starts
    const int64_t t0 = s_tile[0];
    if (t0 < a.num_tiles && is_bulk(t0)) {
      if (!mbar_wait_bounded(&bar[0], 0, a.timeout_ns)) {
        set_error(a.hdr, AK_ERR_TIMEOUT);
        *s_flag = 1;
      }
      phase_bits ^= 1u;
    }
  }
  __syncthreads();

  const int shift = a.pass * RADIX_BITS;
  const uint32_t lt_mask = lanemask_lt();
  const uint32_t gt_mask = ~(lt_mask | (1u << lane));
  uint32_t *wm = wmask + warp * HROW;
  unsigned long long *wm2 = wmask2 + warp * HROW;
  S *st = reinterpret_cast<S *>(a.status_cur);

  for (int it = 0;; ++it) {
    const int s = it % STAGES;
    const int64_t tile = s_tile[s];
    if (tile >= a.num_tiles || *s_flag) break;  // uniform: read after a barrier
    const int64_t base = tile * TILE;
    const int tile_n = int((a.n - base) < int64_t(TILE) ? (a.n - base) : int64_t(TILE));
    U *sk = stage_keys(s);
    V *sv = stage_vals(s);
    if (!is_bulk(tile)) {  // ragged last tile or unaligned source: plain loads
      for (int i = tid; i < tile_n; i += BLOCK) sk[i] = ksrc[base + i];
      if (load_v)
        for (int i = tid; i < tile_n; i += BLOCK) sv[i] = vsrc[base + i];
      __syncthreads();
    }

    // ---- warp multisplit ranking (item i of lane l sits at wbase + 32 i + l)
    const int wbase = warp * 32 * ITEMS;
    uint32_t dr[ITEMS];  // rank << 9 | digit (digit RADIX marks a padding slot)
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int idx = wbase + i * 32 + lane;
      dr[i] = (idx < tile_n) ? pass_digit<DIGIT, KIND>(a, sk[idx], shift) : uint32_t(RADIX);
    }
#if AK_WARP_MATCH == 3
    // two items per step: lane l sets bit l (item A) and bit 32 + l (item B) of
    // the 64-bit mask of its digit; one read gives both peer sets and how many
    // lanes of item A (all earlier than item B) share item B's digit.  Each
    // digit's counter is advanced by exactly one leader: A's group leader, or
    // B's when no lane of A has that digit.
#pragma unroll
    for (int i = 0; i + 1 < ITEMS; i += 2) {
      const uint32_t dA = dr[i], dB = dr[i + 1];
      uint16_t *cA = whist + dA * (2 * L::HSTRIDE) + warp;
      uint16_t *cB = whist + dB * (2 * L::HSTRIDE) + warp;
      atomicOr(&wm2[dA], 1ull << lane);
      atomicOr(&wm2[dB], 1ull << (32 + lane));
      __syncwarp();
      const unsigned long long MA = wm2[dA], MB = wm2[dB];
      const uint32_t nA = *cA, nB = *cB;
      __syncwarp();
      const uint32_t peersA = uint32_t(MA), peersB = uint32_t(MB >> 32), aInB = uint32_t(MB);
      if ((peersA & gt_mask) == 0) {
        *cA = uint16_t(nA + __popcll(MA));
        wm2[dA] = 0ull;
      }
      if (aInB == 0u && (peersB & gt_mask) == 0) {
        *cB = uint16_t(nB + __popc(peersB));
        wm2[dB] = 0ull;
      }
      __syncwarp();
      dr[i] = ((nA + __popc(peersA & lt_mask)) << 9) | dA;
      dr[i + 1] = ((nB + __popc(aInB) + __popc(peersB & lt_mask)) << 9) | dB;
    }
    if (ITEMS & 1) {  // odd item count: the last item alone
      const uint32_t d = dr[ITEMS - 1];
      uint16_t *wc = whist + d * (2 * L::HSTRIDE) + warp;
      atomicOr(&wm2[d], 1ull << lane);
      __syncwarp();
      const uint32_t peers = uint32_t(wm2[d]);
      const uint32_t cnt = *wc;
      __syncwarp();
      if ((peers & gt_mask) == 0) {
        *wc = uint16_t(cnt + __popc(peers));
        wm2[d] = 0ull;
      }
      __syncwarp();
      dr[ITEMS - 1] = ((cnt + __popc(peers & lt_mask)) << 9) | d;
    }
#else
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t d = dr[i];
#if AK_WARP_MATCH == 2
      uint16_t *wc = whist + d * (2 * L::HSTRIDE) + warp;  // this warp's running count of digit d
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
#else
      uint16_t *wc = whist + d * (2 * L::HSTRIDE) + warp;
      const uint32_t peers = warp_peers(d, tile_n != TILE);
      const bool leader = (peers & gt_mask) == 0;  // highest lane of the group
      uint32_t cnt = 0;
      if (leader) cnt = *wc;
      if (leader) *wc = uint16_t(cnt + __popc(peers));
      cnt = __shfl_sync(0xffffffffu, cnt, 31 - __clz(peers));
      __syncwarp();
#endif
      dr[i] = ((cnt + __popc(peers & lt_mask)) << 9) | d;
    }
#endif
    __syncthreads();  // A: every warp row complete

    // ---- per-digit tile counts, publish, warp bases = tile digit start + earlier warps
    uint32_t my_cnt = 0;
    uint32_t *hrow = reinterpret_cast<uint32_t *>(whist) + tid * L::HSTRIDE;
    if (tid < RADIX) {
#pragma unroll
      for (int v = 0; v < NW / 2; ++v) {
        const uint32_t q = hrow[v];
        my_cnt += (q & 0xFFFFu) + (q >> 16);
      }
      const S word = (S(tile == 0 ? FLAG_INC : FLAG_AGG) << StatusWord<S>::SHIFT) | S(my_cnt);
      st_relaxed(&st[tile * RADIX + tid], word);
    }
    uint32_t total;
    const uint32_t start = block_exclusive_scan<BLOCK>(tid < RADIX ? my_cnt : 0u, s_scr, &total);
    if (tid < RADIX) {  // each warp's base = tile digit start + counts of earlier warps
      uint32_t run = start;
#pragma unroll
      for (int v = 0; v < NW / 2; ++v) {
        const uint32_t q = hrow[v];
        const uint32_t lo = run, hi = run + (q & 0xFFFFu);
        run = hi + (q >> 16);
        hrow[v] = (lo & 0xFFFFu) | (hi << 16);
      }
    }
    __syncthreads();  // B

    // ---- scatter the stage into the output buffer in digit order
    U *ok = reinterpret_cast<U *>(smem + L::OFF_OUT);
    V *ov = reinterpret_cast<V *>(smem + L::OFF_OUT + L::KEYS);
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t d = dr[i] & 511u;
      if (d < RADIX) {
        const int idx = wbase + i * 32 + lane;
        const uint32_t pos = uint32_t(whist[d * (2 * L::HSTRIDE) + warp]) + (dr[i] >> 9);
        ok[pos] = sk[idx];
        if (HAS_V) ov[pos] = gen_index ? V(base + idx) : sv[idx];
        if (DIGIT == DIGIT_LEARNED) s_dig[pos] = uint8_t(d);
      }
    }

    // ---- decoupled look-back over a window of predecessors per probe
    if (tid < RADIX) {
      unsigned long long excl = 0;
      if (tile > 0) {
        int64_t j = tile - 1;
        uint64_t t0 = 0;
        uint32_t spins = 0;
        bool done = false;
        while (!done) {
          S w4[LOOKBACK_WINDOW];
#pragma unroll
          for (int k = 0; k < LOOKBACK_WINDOW; ++k)
            w4[k] = (j - k >= 0) ? ld_relaxed(&st[(j - k) * RADIX + tid]) : S(0);
          int used = 0;
#pragma unroll
          for (int k = 0; k < LOOKBACK_WINDOW; ++k) {
            if (done || used != k) break;
            const uint32_t flag = uint32_t(w4[k] >> StatusWord<S>::SHIFT);
            if (flag == 0) break;
            excl += (unsigned long long)(w4[k] & StatusWord<S>::MASK);
            ++used;
            if (flag == FLAG_INC || j - k == 0) done = true;
          }
          j -= used;
          if (!done && used == 0) {
            __nanosleep(64);  // predecessor not published yet: yield issue slots
            if ((++spins & 31u) == 0) {
              const uint64_t now = globaltimer_ns();
              if (t0 == 0) t0 = now;
              else if (now - t0 > a.timeout_ns) {
                set_error(a.hdr, AK_ERR_TIMEOUT);
                done = true;
              }
            }
          }
        }
        const S word = (S(FLAG_INC) << StatusWord<S>::SHIFT) | S(excl + my_cnt);
        st_relaxed(&st[tile * RADIX + tid], word);
      }
      const long long delta = (long long)(a.plan->bin_off[a.pass][tid] + excl) - (long long)start;
      s_kptr[tid] = reinterpret_cast<unsigned long long>(kdst) + (unsigned long long)(delta * (long long)sizeof(U));
      if (HAS_V)
        s_vptr[tid] = reinterpret_cast<unsigned long long>(vdst) + (unsigned long long)(delta * (long long)sizeof(V));
    }
    __syncthreads();  // C
    if (PERSIST)  // counters of the next tile (barrier D follows before its ranking)
      for (int i = tid; i < HROW * L::HSTRIDE; i += BLOCK) reinterpret_cast<uint32_t *>(whist)[i] = 0u;

    // ---- write the tile out: consecutive threads store consecutive keys of a digit run
    if (tile_n == TILE) {
#pragma unroll 4
      for (int r = 0; r < ITEMS; ++r) {
        const int i = r * BLOCK + tid;
        const U k = ok[i];
        const uint32_t d = DIGIT == DIGIT_LEARNED ? uint32_t(s_dig[i]) : digit_of(radix_key_t<KIND>(k, a.flip), shift);
        if (write_keys) reinterpret_cast<U *>(s_kptr[d])[i] = k;
        if (HAS_V) reinterpret_cast<V *>(s_vptr[d])[i] = ov[i];
      }
    } else {
      for (int i = tid; i < tile_n; i += BLOCK) {
        const U k = ok[i];
        const uint32_t d = DIGIT == DIGIT_LEARNED ? uint32_t(s_dig[i]) : digit_of(radix_key_t<KIND>(k, a.flip), shift);
        if (write_keys) reinterpret_cast<U *>(s_kptr[d])[i] = k;
        if (HAS_V) reinterpret_cast<V *>(s_vptr[d])[i] = ov[i];
      }
    }

    if (!PERSIST) break;  // one tile per CTA

    // ---- make the next stage resident, then recycle this one
    if (tid == 0) {
      const int sn = (it + 1) % STAGES;
      const int64_t tn = s_tile[sn];
      if (tn < a.num_tiles && is_bulk(tn)) {
        if (!mbar_wait_bounded(&bar[sn], (phase_bits >> sn) & 1u, a.timeout_ns)) {
          set_error(a.hdr, AK_ERR_TIMEOUT);
          *s_flag = 1;
        }
        phase_bits ^= 1u << sn;
      }
    }
    __syncthreads();  // D: stage s is free, the next stage is resident
    if (tid == 0 && !*s_flag) {
      const int64_t t = next_tile();
      s_tile[s] = uint32_t(t < a.num_tiles ? t : a.num_tiles);
      issue(s, t);
    }
    // s_tile[s] is next read STAGES-1 iterations later, after barriers
  }
  // a copy left in flight by a timed-out wait must land before the CTA exits
  if (tid == 0 && *s_flag) {
    for (int s = 0; s < STAGES; ++s) mbar_wait_bounded(&bar[s], (phase_bits >> s) & 1u, a.timeout_ns);
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
