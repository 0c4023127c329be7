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
};

// ------------------------------------------------------------------ histogram
template <typename U, int BLOCK>
__global__ void __launch_bounds__(BLOCK) hist_kernel(const U *__restrict__ keys, int64_t n, int kind,
                                                     U flip, unsigned long long *counts,
                                                     uint4 *zero_buf, int64_t zero_vec) {
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
                                                     int path_tag) {
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
template <typename U, typename V, int BLOCK, int ITEMS, bool HAS_V>
struct PassSmem {
  static constexpr int TILE = BLOCK * ITEMS;
  static constexpr int NW = BLOCK / 32;
  static constexpr size_t KEYS = size_t(TILE) * sizeof(U);
  static constexpr size_t VALS = HAS_V ? size_t(TILE) * sizeof(V) : 0;
  static constexpr size_t OFF_V = KEYS;                                  // 16-aligned
  static constexpr size_t OFF_HIST = (OFF_V + VALS + 15) / 16 * 16;
  static constexpr size_t OFF_DELTA = OFF_HIST + size_t(NW) * RADIX * 4;  // int64[RADIX]
  static constexpr size_t OFF_START = OFF_DELTA + RADIX * 8;              // u32[RADIX]
  static constexpr size_t OFF_SCR = OFF_START + RADIX * 4;                // u32[NW+1]
  static constexpr size_t OFF_BAR = (OFF_SCR + (NW + 1) * 4 + 15) / 16 * 16;
  static constexpr size_t OFF_TILE = OFF_BAR + 8;
  static constexpr size_t BYTES = OFF_TILE + 8;
};

template <typename U, typename V, typename S, int BLOCK, int ITEMS, bool HAS_V>
__global__ void __launch_bounds__(BLOCK) onesweep_pass(PassArgs<U, V> a) {
  using L = PassSmem<U, V, BLOCK, ITEMS, HAS_V>;
  constexpr int TILE = L::TILE;
  constexpr int NW = L::NW;
  static_assert(BLOCK >= RADIX, "one digit per thread in the look-back");
  extern __shared__ __align__(128) uint8_t smem[];
  U *sk = reinterpret_cast<U *>(smem);
  V *sv = reinterpret_cast<V *>(smem + L::OFF_V);
  uint32_t *whist = reinterpret_cast<uint32_t *>(smem + L::OFF_HIST);
  long long *s_delta = reinterpret_cast<long long *>(smem + L::OFF_DELTA);
  uint32_t *s_start = reinterpret_cast<uint32_t *>(smem + L::OFF_START);
  uint32_t *s_scr = reinterpret_cast<uint32_t *>(smem + L::OFF_SCR);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::OFF_BAR);
  uint32_t *s_tile = reinterpret_cast<uint32_t *>(smem + L::OFF_TILE);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // The next pass's look-back words: each launch of this kernel has exactly
  // num_tiles CTAs, so block b clears row b.
  if (a.status_next) {
    S *nx = reinterpret_cast<S *>(a.status_next) + int64_t(blockIdx.x) * RADIX;
    for (int i = tid; i < RADIX; i += BLOCK) nx[i] = S(0);
  }
  const uint32_t q = a.plan->q[a.pass];
  if (q == INACTIVE) return;
  const uint32_t m = a.plan->m;

  for (int i = tid; i < NW * RADIX; i += BLOCK) whist[i] = 0;
  if (tid == 0) {
    *s_tile = atomicAdd(&a.hdr->tile_counter[a.pass], 1u) + (a.debug_skip ? 1u : 0u);
    mbar_init(bar, 1);
  }
  __syncthreads();
  const int64_t tile = *s_tile;
  __syncthreads();  // s_tile is reused below as the bulk-copy verdict
  if (tile >= a.num_tiles) return;  // only under the test hook
  const int64_t base = tile * TILE;
  const int tile_n = int((a.n - base) < int64_t(TILE) ? (a.n - base) : int64_t(TILE));

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

  // ---- stage the tile in shared memory
  const bool load_v = HAS_V && !gen_index;
  const bool bulk = (tile_n == TILE) &&
                    ((reinterpret_cast<uintptr_t>(ksrc + base) & 15) == 0) &&
                    (!load_v || ((reinterpret_cast<uintptr_t>(vsrc + base) & 15) == 0));
  if (bulk) {
    // one thread issues and waits (bounded); the verdict is shared so that the
    // whole CTA takes the same branch
    if (tid == 0) {
      mbar_expect_tx(bar, uint32_t(L::KEYS + (load_v ? L::VALS : 0)));
      bulk_g2s(sk, ksrc + base, uint32_t(L::KEYS), bar);
      if (load_v) bulk_g2s(sv, vsrc + base, uint32_t(L::VALS), bar);
      uint32_t ok = mbar_wait_bounded(bar, 0, a.timeout_ns) ? 1u : 0u;
      if (!ok) {
        set_error(a.hdr, AK_ERR_TIMEOUT);
        mbar_wait_bounded(bar, 0, a.timeout_ns);  // let the copy land before exiting
      }
      *s_tile = ok;  // tile id already read by every thread
    }
    __syncthreads();
    if (*s_tile == 0) return;
    while (!mbar_try_wait(bar, 0)) {
    }  // phase already complete: observes the async-proxy writes
  } else {
    for (int i = tid; i < tile_n; i += BLOCK) sk[i] = ksrc[base + i];
    if (load_v)
      for (int i = tid; i < tile_n; i += BLOCK) sv[i] = vsrc[base + i];
    __syncthreads();
  }

  // ---- warp multisplit ranking (warp-striped: item i of lane l is at wbase+32i+l)
  const int shift = a.pass * RADIX_BITS;
  const int wbase = warp * 32 * ITEMS;
  U keys[ITEMS];
  uint32_t rank[ITEMS];
  V vals[HAS_V ? ITEMS : 1];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int idx = wbase + i * 32 + lane;
    keys[i] = (idx < tile_n) ? sk[idx] : U(0);
    if (HAS_V) {
      if (gen_index) vals[i] = V(base + idx);
      else vals[i] = (idx < tile_n) ? sv[idx] : V(0);
    }
  }
  uint32_t *wh = whist + warp * RADIX;
  const uint32_t lt_mask = lanemask_lt();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int idx = wbase + i * 32 + lane;
    const bool valid = idx < tile_n;
    const uint32_t d = valid ? digit_of(radix_key(keys[i], a.kind, a.flip), shift) : 0xFFFFFFFFu;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int leader = 31 - __clz(peers);
    uint32_t cnt = 0;
    if (lane == leader && valid) {
      cnt = wh[d];
      wh[d] = cnt + __popc(peers);
    }
    __syncwarp();
    cnt = __shfl_sync(0xffffffffu, cnt, leader);
    rank[i] = cnt + __popc(peers & lt_mask);
  }
  __syncthreads();

  // ---- per-digit tile counts, publish, tile-local digit starts
  uint32_t my_cnt = 0;
  S *st = reinterpret_cast<S *>(a.status_cur);
  if (tid < RADIX) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = whist[w * RADIX + tid];
      whist[w * RADIX + tid] = run;
      run += c;
    }
    my_cnt = run;
    const S word = (S(tile == 0 ? FLAG_INC : FLAG_AGG) << StatusWord<S>::SHIFT) | S(my_cnt);
    st_relaxed(&st[tile * RADIX + tid], word);
  }
  uint32_t total;
  const uint32_t start = block_exclusive_scan<BLOCK>(tid < RADIX ? my_cnt : 0u, s_scr, &total);
  if (tid < RADIX) s_start[tid] = start;
  __syncthreads();

  // ---- scatter into shared memory in digit order (all reads of sk/sv are done)
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int idx = wbase + i * 32 + lane;
    if (idx < tile_n) {
      const uint32_t d = digit_of(radix_key(keys[i], a.kind, a.flip), shift);
      const uint32_t pos = s_start[d] + wh[d] + rank[i];
      sk[pos] = keys[i];
      if (HAS_V) sv[pos] = vals[i];
    }
  }

  // ---- decoupled look-back: exclusive prefix of this digit over earlier tiles
  if (tid < RADIX) {
    unsigned long long excl = 0;
    if (tile > 0) {
      int64_t j = tile - 1;
      uint64_t t0 = 0;
      uint32_t spins = 0;
      while (true) {
        const S v = ld_relaxed(&st[j * RADIX + tid]);
        const uint32_t flag = uint32_t(v >> StatusWord<S>::SHIFT);
        if (flag == 0) {
          if ((++spins & 63u) == 0) {
            const uint64_t now = globaltimer_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > a.timeout_ns) {
              set_error(a.hdr, AK_ERR_TIMEOUT);
              break;
            }
          }
          continue;
        }
        excl += (unsigned long long)(v & StatusWord<S>::MASK);
        if (flag == FLAG_INC || j == 0) break;
        --j;
      }
      const S word = (S(FLAG_INC) << StatusWord<S>::SHIFT) | S(excl + my_cnt);
      st_relaxed(&st[tile * RADIX + tid], word);
    }
    s_delta[tid] = (long long)(a.plan->bin_off[a.pass][tid] + excl) - (long long)s_start[tid];
  }
  __syncthreads();

  // ---- write the tile out: consecutive threads store consecutive keys of a digit run
  for (int i = tid; i < tile_n; i += BLOCK) {
    const U k = sk[i];
    const long long g = s_delta[digit_of(radix_key(k, a.kind, a.flip), shift)] + i;
    if (write_keys) kdst[g] = k;
    if (HAS_V) vdst[g] = sv[i];
  }
}

// --------------------------------------------------------------------- finish
template <typename U, typename V, bool HAS_V>
__global__ void finish_kernel(PassArgs<U, V> a) {
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
