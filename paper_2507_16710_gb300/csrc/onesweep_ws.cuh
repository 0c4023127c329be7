// onesweep_ws.cuh -- digit pass with a dedicated look-back warp.
//
// Same contract as onesweep_pass (one stable LSD pass of an 8-bit digit, tiles
// claimed in increasing order, decoupled look-back over predecessor tiles), with
// the work split between two kinds of warps so that the look-back's waiting is
// off the path of the data:
//
//   compute warps (NCW of them)   per tile t_j:
//     1. keys (and values) of t_j from its shared tile buffer (filled by a bulk
//        copy issued one tile ahead) into registers; digits
//     2. warp multisplit ranking (peer masks, per-warp 16-bit digit counters)
//     3. per-digit tile counts: published to the look-back words (flag AGG),
//        handed to the look-back warp; the next tile is claimed and its bulk
//        copy issued into a free buffer; digit starts and warp bases
//     4. scatter of t_j into digit order in its own tile buffer (the keys are
//        in registers, so the buffer that staged them is free)
//     5. write-out of t_{j-1}, whose destinations the look-back warp has had a
//        whole tile's time to find
//   look-back warp               per tile t_j, as soon as its counts arrive:
//     8 digits per lane: digit starts, look-back over windows of predecessors,
//     inclusive counts published (flag INC), per-digit destination of the
//     tile's first output slot for the write-out.
//
// Three tile buffers rotate (t_{j+1} landing, t_j ranked and scattered, t_{j-1}
// written out); two slots of per-digit state alternate between the compute
// warps and the look-back warp, handed over through mbarriers.  Every wait is
// bounded by timeout_ns: an expired wait records AK_ERR_TIMEOUT in the status
// word, skips the stores that would depend on it and ends the CTA after its
// bulk copies have landed.  No trap.
#pragma once

#include "internal.h"
#include "onesweep.cuh"

namespace ak {

// Peer matching of the warp multisplit: which lanes of the warp hold the same
// digit as this lane.
enum WsRank : int {
  WS_RANK_BALLOT = 0,  // one warp vote per digit bit: no shared memory
  WS_RANK_OR = 1,      // lanes OR their bit into a per-warp shared word per digit
  WS_RANK_MATCH = 2    // the match.any warp instruction
};
// predecessors probed per look-back round trip (8 status words of each per lane)
template <typename S> constexpr int ws_lb_win() { return sizeof(S) == 4 ? 4 : 2; }

template <typename U, typename V, bool HAS_V, int ITEMS, int RANK>
struct WsSmem {
  static constexpr int TILE = WS_NC * ITEMS;
  static constexpr int HW = 16;               // warp columns per digit row (15 used)
  static constexpr int HSTRIDE = HW / 2 + 1;  // 32-bit words per digit row (odd: rows start in different banks)
  static constexpr int H2 = 2 * HSTRIDE;      // u16 slots per digit row
  static constexpr int HROW = RADIX + 1;      // digit rows + the padding digit of a ragged tile
  static constexpr size_t KEYS = size_t(TILE) * sizeof(U);
  static constexpr size_t VALS = HAS_V ? size_t(TILE) * sizeof(V) : 0;
  static constexpr size_t BUF = (KEYS + VALS + 127) / 128 * 128;
  static constexpr size_t OFF_DIG = 3 * BUF;                                        // u8[2][TILE]
  static constexpr size_t OFF_HIST = OFF_DIG + (2 * size_t(TILE) + 15) / 16 * 16;   // u32[HROW][HSTRIDE]
  static constexpr size_t OFF_MASK = OFF_HIST + (size_t(HROW) * HSTRIDE * 4 + 15) / 16 * 16;  // u32[NCW][HROW]
  static constexpr size_t MASK_BYTES = RANK == WS_RANK_OR ? (size_t(WS_NCW) * HROW * 4 + 15) / 16 * 16 : 0;
  static constexpr size_t OFF_BIN = OFF_MASK + MASK_BYTES;      // i64[RADIX]: digit offsets of the pass
  static constexpr size_t OFF_CNT = OFF_BIN + RADIX * 8;        // u32[2][RADIX]: tile counts -> look-back warp
  static constexpr size_t OFF_DELTA = OFF_CNT + 2 * RADIX * 4;  // [2][RADIX] 8-byte slots: destination of slot 0
  static constexpr size_t OFF_SCR = OFF_DELTA + 2 * RADIX * 8;  // u32[RADIX / 32]: warp totals of the digit scan
  static constexpr size_t OFF_BAR = OFF_SCR + 32;               // u64: stage, cnt[2], lb[2]
  static constexpr size_t OFF_LBT = OFF_BAR + 5 * 8;            // i64[2]: tile of each look-back slot (-1: end)
  static constexpr size_t OFF_NEXT = OFF_LBT + 16;              // i64: next tile
  static constexpr size_t OFF_ABORT = OFF_NEXT + 8;             // u32
  static constexpr size_t BYTES = OFF_ABORT + 16;
  static_assert(BYTES == ws_smem_bytes(int(sizeof(U)), HAS_V ? int(sizeof(V)) : 0, ITEMS, RANK == WS_RANK_OR),
                "host-side size of the shared memory");
  static_assert(TILE < 65536, "warp bases are u16");
  static_assert(KEYS % 16 == 0 && BUF % 128 == 0 && OFF_BIN % 8 == 0 && OFF_DELTA % 8 == 0 && OFF_BAR % 8 == 0,
                "shared-memory arrays aligned to their element size (bulk copies: 16 bytes)");
};

__device__ __forceinline__ void mbar_arrive_cnt(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Eight consecutive look-back words (8-digit group of one lane), relaxed.
__device__ __forceinline__ void ld_relaxed_8(const uint32_t *p, uint32_t (&w)[8]) {
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
               : "l"(p)
               : "memory");
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
               : "l"(p + 4)
               : "memory");
}
__device__ __forceinline__ void ld_relaxed_8(const unsigned long long *p, unsigned long long (&w)[8]) {
#pragma unroll
  for (int h = 0; h < 4; ++h)
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0,%1}, [%2];"
                 : "=l"(w[2 * h]), "=l"(w[2 * h + 1])
                 : "l"(p + 2 * h)
                 : "memory");
}
__device__ __forceinline__ void st_relaxed_8(uint32_t *p, const uint32_t (&w)[8]) {
  asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]),
               "r"(w[3])
               : "memory");
  asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p + 4), "r"(w[4]), "r"(w[5]), "r"(w[6]),
               "r"(w[7])
               : "memory");
}
__device__ __forceinline__ void st_relaxed_8(unsigned long long *p, const unsigned long long (&w)[8]) {
#pragma unroll
  for (int h = 0; h < 4; ++h)
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1,%2};" ::"l"(p + 2 * h), "l"(w[2 * h]), "l"(w[2 * h + 1])
                 : "memory");
}

template <typename U, typename V, bool HAS_V, int KIND, typename S, int ITEMS, int DIGIT = DIGIT_RADIX,
          int RANK = AK_WS_RANK>
__global__ void __launch_bounds__(WS_BLOCK, 2) onesweep_ws_pass(PassArgs<U, V> a) {
  using L = WsSmem<U, V, HAS_V, ITEMS, RANK>;
  constexpr int TILE = L::TILE;
  constexpr int H2 = L::H2;
  constexpr int HROW = L::HROW;
  static_assert(DIGIT != DIGIT_VALUE || HAS_V, "a value-carried digit needs the value stream");
  using Delta = typename std::conditional<sizeof(S) == 4, int32_t, long long>::type;
  extern __shared__ __align__(128) uint8_t smem[];
  uint16_t *whist = reinterpret_cast<uint16_t *>(smem + L::OFF_HIST);
  uint32_t *whist32 = reinterpret_cast<uint32_t *>(smem + L::OFF_HIST);
  long long *s_bin = reinterpret_cast<long long *>(smem + L::OFF_BIN);
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + L::OFF_CNT);
  Delta *s_delta = reinterpret_cast<Delta *>(smem + L::OFF_DELTA);  // [2][RADIX], 8-byte slots
  uint32_t *s_scr = reinterpret_cast<uint32_t *>(smem + L::OFF_SCR);
  uint64_t *bar_stage = reinterpret_cast<uint64_t *>(smem + L::OFF_BAR);
  uint64_t *bar_cnt = bar_stage + 1;  // [2]: tile counts handed to the look-back warp
  uint64_t *bar_lb = bar_stage + 3;   // [2]: destinations handed back
  long long *s_lbt = reinterpret_cast<long long *>(smem + L::OFF_LBT);
  long long *s_next = reinterpret_cast<long long *>(smem + L::OFF_NEXT);
  uint32_t *s_abort = reinterpret_cast<uint32_t *>(smem + L::OFF_ABORT);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (a.gate && *a.gate != a.gate_want) return;

  // Clear the next pass's look-back rows (the grid covers rows blockIdx.x + k*gridDim.x).
  if (a.status_next) {
    S *nx = reinterpret_cast<S *>(a.status_next);
    for (int64_t r = blockIdx.x; r < a.num_tiles; r += gridDim.x)
      for (int i = tid; i < RADIX; i += WS_BLOCK) nx[r * RADIX + i] = S(0);
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
  const int64_t full_tiles = a.n / TILE;
  auto is_bulk = [&](int64_t t) { return aligned && t < full_tiles; };
  auto buf_k = [&](int b) { return reinterpret_cast<U *>(smem + size_t(b) * L::BUF); };
  auto buf_v = [&](int b) { return reinterpret_cast<V *>(smem + size_t(b) * L::BUF + L::KEYS); };
  auto dig_of = [&](int s) { return smem + L::OFF_DIG + size_t(s) * TILE; };
  auto claim = [&]() -> int64_t {
    const int64_t t = int64_t(atomicAdd(&a.hdr->tile_counter[a.pass], 1u)) + (a.debug_skip ? 1 : 0);
    return t < a.num_tiles ? t : a.num_tiles;
  };
  auto issue = [&](int64_t t, int b) {  // one thread; buffer b must be free
    mbar_expect_tx(bar_stage, uint32_t(L::KEYS + (load_v ? L::VALS : 0)));
    bulk_g2s(buf_k(b), ksrc + t * TILE, uint32_t(L::KEYS), bar_stage);
    if (load_v) bulk_g2s(buf_v(b), vsrc + t * TILE, uint32_t(L::VALS), bar_stage);
  };

  for (int i = tid; i < HROW * L::HSTRIDE; i += WS_BLOCK) whist32[i] = 0u;
  if constexpr (RANK == WS_RANK_OR) {
    uint32_t *wmask = reinterpret_cast<uint32_t *>(smem + L::OFF_MASK);
    for (int i = tid; i < WS_NCW * HROW; i += WS_BLOCK) wmask[i] = 0u;
  }
  for (int i = tid; i < RADIX; i += WS_BLOCK) s_bin[i] = (long long)a.plan->bin_off[a.pass][i];
  if (tid == 0) {
    mbar_init(bar_stage, 1);
    mbar_init(bar_cnt, RADIX);
    mbar_init(bar_cnt + 1, RADIX);
    mbar_init(bar_lb, 32);
    mbar_init(bar_lb + 1, 32);
    *s_abort = 0;
    const int64_t t = claim();
    *s_next = (long long)t;
    if (t < a.num_tiles && is_bulk(t)) issue(t, 0);
  }
  __syncthreads();
  S *st = reinterpret_cast<S *>(a.status_cur);
  const int shift = a.pass * RADIX_BITS;

  if (warp == WS_NCW) {
    // =============================== look-back warp ===============================
    // lane owns digits 8*lane .. 8*lane+7
    for (uint32_t k = 0;; ++k) {
      const uint32_t slot = k & 1u, par = (k >> 1) & 1u;
      // every lane waits; the warp goes on together or stops together (shuffles follow)
      const bool got = mbar_wait_bounded(bar_cnt + slot, par, a.timeout_ns);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) set_error(a.hdr, AK_ERR_TIMEOUT);
        break;
      }
      const long long tile = s_lbt[slot];
      if (tile < 0) break;
      const uint32_t *cnt = s_cnt + slot * RADIX + 8 * lane;  // re-read where needed (registers)
      uint32_t tot = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) tot += cnt[j];
      const uint32_t lane_start = warp_inclusive_scan(tot) - tot;
      using Acc = typename std::conditional<sizeof(S) == 4, uint32_t, unsigned long long>::type;
      constexpr int WIN = ws_lb_win<S>();
      Acc excl[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) excl[j] = 0;
      if (tile > 0) {
        int64_t p = tile - 1;
        uint32_t done = 0;  // bit j: digit 8*lane+j found an inclusive predecessor
        uint64_t t0 = 0;
        uint32_t spins = 0;
        for (;;) {
          S w[WIN][8];
#pragma unroll
          for (int r = 0; r < WIN; ++r) {
            if (p - r >= 0) {
              ld_relaxed_8(&st[(p - r) * RADIX + 8 * lane], w[r]);
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) w[r][j] = S(0);
            }
          }
          int used = 0;
          bool stop = false;
#pragma unroll
          for (int r = 0; r < WIN; ++r) {
            if (!stop) {
              bool ready = true;
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (!((done >> j) & 1u) && (w[r][j] >> StatusWord<S>::SHIFT) == 0) ready = false;
              if (!ready) {
                stop = true;  // a digit of predecessor p - r is not published yet
              } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  if (!((done >> j) & 1u)) {
                    excl[j] += Acc(w[r][j] & StatusWord<S>::MASK);
                    if (uint32_t(w[r][j] >> StatusWord<S>::SHIFT) == FLAG_INC) done |= 1u << j;
                  }
                }
                ++used;
                if (done == 0xFFu) stop = true;
              }
            }
          }
          if (done == 0xFFu) break;
          p -= used;
          if (used == 0) {
            __nanosleep(64);
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
        S out[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] = (S(FLAG_INC) << StatusWord<S>::SHIFT) | S(excl[j] + cnt[j]);
        st_relaxed_8(&st[tile * RADIX + 8 * lane], out);
      }
      uint32_t run = lane_start;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int d = 8 * lane + j;
        s_delta[slot * RADIX + d] = Delta(s_bin[d] + (long long)excl[j] - (long long)run);
        run += cnt[j];
      }
      mbar_arrive_cnt(bar_lb + slot, 1);  // each lane after its own stores
    }
    return;
  }

  // ================================ compute warps ================================
  const uint32_t lt_mask = lanemask_lt();
  const uint32_t gt_mask = ~(lt_mask | (1u << lane));
  uint32_t sphase = 0;  // parity of the next completion of bar_stage
  bool pending = false;  // a bulk copy was issued and not yet waited for
  {
    const int64_t t = *s_next;
    pending = t < a.num_tiles && is_bulk(t);
  }
  int64_t prev_tile = -1;
  int prev_n = 0;
  bool aborted = false;

  // write-out of the tile ranked in iteration jj (buffer jj % 3, digit/delta slot jj & 1)
  auto write_out = [&](uint32_t jj, int tile_n) {
    const U *ok = buf_k(int(jj % 3u));
    const V *ov = buf_v(int(jj % 3u));
    const uint8_t *dg = dig_of(int(jj & 1u));
    const Delta *dl = s_delta + (jj & 1u) * RADIX;
    if (tile_n == TILE) {
      constexpr int WB = ITEMS % 4 == 0 ? 4 : (ITEMS % 3 == 0 ? 3 : (ITEMS % 2 == 0 ? 2 : 1));
#pragma unroll
      for (int r0 = 0; r0 < ITEMS; r0 += WB) {
        U k[WB];
        Delta dst[WB];
#pragma unroll
        for (int r = 0; r < WB; ++r) {
          const int i = (r0 + r) * WS_NC + tid;
          k[r] = ok[i];
          dst[r] = dl[dg[i]] + Delta(i);
        }
#pragma unroll
        for (int r = 0; r < WB; ++r) {
          if (write_keys) kdst[dst[r]] = k[r];
          if (HAS_V) vdst[dst[r]] = ov[(r0 + r) * WS_NC + tid];
        }
      }
    } else {
      for (int i = tid; i < tile_n; i += WS_NC) {
        const Delta dst = dl[dg[i]] + Delta(i);
        if (write_keys) kdst[dst] = ok[i];
        if (HAS_V) vdst[dst] = ov[i];
      }
    }
  };

  uint32_t j = 0;
  for (;; ++j) {
    const int64_t tile = *s_next;  // written before barrier C7 of the previous iteration (or the start)
    if (tile >= a.num_tiles) break;
    const int b = int(j % 3u);
    const int slot = int(j & 1u);
    const int64_t base = tile * TILE;
    const int tile_n = int((a.n - base) < int64_t(TILE) ? (a.n - base) : int64_t(TILE));
    const bool bulk = is_bulk(tile);
    bool stage_ok = true;
    if (bulk) {
      if (mbar_wait_bounded(bar_stage, sphase, a.timeout_ns)) {
        pending = false;
        sphase ^= 1u;
      } else {  // the copy is still owed: the exit path waits for it again
        set_error(a.hdr, AK_ERR_TIMEOUT);
        *s_abort = 1;
        stage_ok = false;
      }
    }

    // ---- 1. keys (values) into registers, digits
    const int wbase = warp * 32 * ITEMS;
    U kr[ITEMS];
    V vr[ITEMS];
    uint32_t dr[ITEMS];  // rank << 9 | digit (digit RADIX marks a padding slot)
    {
      const U *sk = buf_k(b);
      const V *sv = buf_v(b);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int idx = wbase + i * 32 + lane;
        const bool valid = idx < tile_n && stage_ok;
        if (valid) {
          kr[i] = bulk ? sk[idx] : ksrc[base + idx];
          if (HAS_V) vr[i] = gen_index ? V(base + idx) : (bulk ? sv[idx] : vsrc[base + idx]);
        } else {
          kr[i] = U(0);
          if (HAS_V) vr[i] = V(0);
        }
        if constexpr (DIGIT == DIGIT_VALUE)
          dr[i] = valid ? ((uint32_t(vr[i]) >> shift) & uint32_t(RADIX - 1)) : uint32_t(RADIX);
        else
          dr[i] = valid ? pass_digit<DIGIT, KIND>(a, kr[i], shift) : uint32_t(RADIX);
      }
    }

    // ---- 2. warp multisplit ranking
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const uint32_t d = dr[i];
      uint32_t peers;
      if constexpr (RANK == WS_RANK_MATCH) {
        peers = __match_any_sync(0xffffffffu, d);
      } else if constexpr (RANK == WS_RANK_OR) {
        uint32_t *wm = reinterpret_cast<uint32_t *>(smem + L::OFF_MASK) + warp * HROW;
        atomicOr(&wm[d], 1u << lane);
        __syncwarp();
        peers = wm[d];
        __syncwarp();
        if ((peers & gt_mask) == 0) wm[d] = 0u;
      } else {
        peers = __ballot_sync(0xffffffffu, d < uint32_t(RADIX));
        if (d >= uint32_t(RADIX)) peers = ~peers;  // padding lanes group together
#pragma unroll
        for (int bit = 0; bit < RADIX_BITS; ++bit) {
          const bool on = (d >> bit) & 1u;
          const uint32_t v = __ballot_sync(0xffffffffu, on);
          peers &= on ? v : ~v;
        }
      }
      uint16_t *wc = whist + d * H2 + warp;  // this warp's running count of digit d
      const uint32_t cnt = *wc;
      __syncwarp();
      if ((peers & gt_mask) == 0) *wc = uint16_t(cnt + __popc(peers));  // highest lane of the group
      __syncwarp();
      dr[i] = ((cnt + __popc(peers & lt_mask)) << 9) | d;
    }
    named_sync(1, WS_NC);  // C5: every warp column complete
    if (*s_abort) {
      aborted = true;
      break;
    }

    // ---- 3. tile counts: publish, hand to the look-back warp; claim the next tile
    uint32_t my_cnt = 0, inc = 0;
    uint32_t *hrow = whist32 + tid * L::HSTRIDE;
    if (tid < RADIX) {
#pragma unroll
      for (int v = 0; v < L::HW / 2; ++v) {
        const uint32_t w = hrow[v];
        my_cnt += (w & 0xFFFFu) + (w >> 16);
      }
      st_relaxed(&st[tile * RADIX + tid], (S(tile == 0 ? FLAG_INC : FLAG_AGG) << StatusWord<S>::SHIFT) | S(my_cnt));
      s_cnt[slot * RADIX + tid] = my_cnt;
      if (tid == 0) s_lbt[slot] = (long long)tile;
      mbar_arrive_cnt(bar_cnt + slot, 1);
      inc = warp_inclusive_scan(my_cnt);
      if (lane == 31) s_scr[warp] = inc;
    } else if (tid == RADIX) {
      const int64_t nt = claim();
      *s_next = (long long)nt;
      if (nt < a.num_tiles && is_bulk(nt)) issue(nt, int((j + 1) % 3u));  // buffer of tile j-2: written out
    }
    named_sync(1, WS_NC);  // C7: warp totals of the digit scan; next tile id
    {
      const int64_t nt = *s_next;
      if (nt < a.num_tiles && is_bulk(nt)) pending = true;
    }
    if (tid < RADIX) {
      uint32_t start = inc - my_cnt;
#pragma unroll
      for (int w2 = 0; w2 < RADIX / 32; ++w2)
        if (w2 < warp) start += s_scr[w2];
      uint32_t run = start;  // warp bases: digit start + counts of earlier warps
#pragma unroll
      for (int v = 0; v < L::HW / 2; ++v) {
        const uint32_t w = hrow[v];
        const uint32_t lo = run, hi = run + (w & 0xFFFFu);
        run = hi + (w >> 16);
        // column WS_NCW belongs to no compute warp: it stays 0, as the next
        // tile's counts sum every column of the row
        hrow[v] = (lo & 0xFFFFu) | (2 * v + 1 < WS_NCW ? (hi << 16) : 0u);
      }
    }
    named_sync(1, WS_NC);  // C9: warp bases ready

    // ---- 4. scatter into digit order in this tile's own buffer
    {
      U *ok = buf_k(b);
      V *ov = buf_v(b);
      uint8_t *dg = dig_of(slot);
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const uint32_t d = dr[i] & 511u;
        if (d < uint32_t(RADIX)) {
          const uint32_t pos = uint32_t(whist[d * H2 + warp]) + (dr[i] >> 9);
          ok[pos] = kr[i];
          if (HAS_V) ov[pos] = vr[i];
          dg[pos] = uint8_t(d);
        }
      }
      __syncwarp();
      for (int dd = lane; dd < HROW; dd += 32) whist[dd * H2 + warp] = 0;  // this warp's column, for the next tile
    }

    // ---- 5. write-out of the previous tile
    if (prev_tile >= 0) {
      if (mbar_wait_bounded(bar_lb + ((j - 1) & 1u), ((j - 1) >> 1) & 1u, a.timeout_ns)) {
        write_out(j - 1, prev_n);
      } else {
        set_error(a.hdr, AK_ERR_TIMEOUT);
        *s_abort = 1;  // every thread stops at the next barrier
      }
    }
    prev_tile = tile;
    prev_n = tile_n;
  }
  if (!aborted && prev_tile >= 0) {  // (uniform: every compute thread left the loop at the same point)
    named_sync(1, WS_NC);  // the last tile's scatter is complete in every warp
    if (mbar_wait_bounded(bar_lb + ((j - 1) & 1u), ((j - 1) >> 1) & 1u, a.timeout_ns)) {
      write_out(j - 1, prev_n);
    } else {
      set_error(a.hdr, AK_ERR_TIMEOUT);
    }
  }
  if (tid == 0) {
    if (!aborted) {  // release the look-back warp
      s_lbt[j & 1u] = -1;
      mbar_arrive_cnt(bar_cnt + (j & 1u), RADIX);
    }
    // a copy left in flight by a timed-out wait must land before the CTA exits
    if (pending) mbar_wait_bounded(bar_stage, sphase, a.timeout_ns);
  }
}

}  // namespace ak
