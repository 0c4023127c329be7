// radix_launch.cuh -- host launch sequence of the onesweep radix sort for one
// key word width and key kind.
#pragma once

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "internal.h"
#include "onesweep.cuh"
#include "onesweep_ws.cuh"

namespace ak {

// Resident CTAs per SM of a kernel launch shape (cached per kernel and device).
template <typename K>
int resident_ctas(K kern, int block, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_pair(reinterpret_cast<const void *>(kern), dev);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, smem) != cudaSuccess || nb < 1) nb = 1;
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = nb;
  return nb;
}

// Digit-pass kernel, its block size, shared memory and tile of a configuration.
template <typename U, typename V, bool HAS_V, int KIND, typename S, int CFG, int DIGIT = DIGIT_RADIX>
struct PassKernel {
  static constexpr int ITEMS = tile_items(sizeof(U), HAS_V ? sizeof(V) : 0, CFG);
  static constexpr int BLOCK = CFG_BLOCK[CFG];
  static constexpr bool PERSIST = CFG_PERSIST[CFG];
  static constexpr int TILE = tile_keys(sizeof(U), HAS_V ? sizeof(V) : 0, CFG);
  static constexpr size_t bytes() {
    if constexpr (CFG == CFG_WS) return WsSmem<U, V, HAS_V, ITEMS, AK_WS_RANK>::BYTES;
    else return PassSmem<U, V, HAS_V, BLOCK, ITEMS>::BYTES;
  }
  static constexpr size_t BYTES = bytes();
  static auto kernel() {
    if constexpr (CFG == CFG_WS) return onesweep_ws_pass<U, V, HAS_V, KIND, S, ITEMS, DIGIT, AK_WS_RANK>;
    else if constexpr (CFG == CFG_RTS) return onesweep_pass<U, V, HAS_V, KIND, S, BLOCK, ITEMS, true, DIGIT, true>;
    else return onesweep_pass<U, V, HAS_V, KIND, S, BLOCK, ITEMS, PERSIST, DIGIT>;
  }
  static_assert(CFG == CFG_WS ? WsSmem<U, V, HAS_V, ITEMS, AK_WS_RANK>::TILE == TILE
                              : PassSmem<U, V, HAS_V, BLOCK, ITEMS>::TILE == TILE,
                "tile shape");
};

template <typename U, typename V, bool HAS_V, int KIND, typename S, int CFG, int DIGIT = DIGIT_RADIX>
cudaError_t run_passes(const RadixCall &c, PassArgs<U, V> a) {
  using P = PassKernel<U, V, HAS_V, KIND, S, CFG, DIGIT>;
  constexpr int BLOCK = P::BLOCK;
  constexpr bool PERSIST = P::PERSIST;
  constexpr int TILE = P::TILE;
  constexpr size_t BYTES = P::BYTES;
  auto kern = P::kernel();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(BYTES));
  if (e != cudaSuccess) return e;
  const int64_t tiles = (c.n + TILE - 1) / TILE;
  a.num_tiles = tiles;
  constexpr int PASSES = sizeof(U);
  const int sms = device_sm_count();
  {  // histogram + zero the first pass's look-back words (reduce-then-scan passes have none)
    constexpr int HB = 256;
    const int64_t want = (c.n + HB * 16 - 1) / (HB * 16);
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 8)));
    const int64_t zero_vec = CFG == CFG_RTS ? 0 : tiles * RADIX * int64_t(sizeof(S)) / 16;
    hist_kernel<U, HB><<<grid, HB, 0, c.stream>>>(reinterpret_cast<const U *>(c.k_in), c.n, c.kind, a.flip,
                                                   c.counts, reinterpret_cast<uint4 *>(c.status[0]), zero_vec,
                                                   c.gate, c.gate_want);
  }
  plan_kernel<<<1, RADIX, 0, c.stream>>>(c.counts, c.n, PASSES, c.plan, c.hdr, c.path_tag, c.gate, c.gate_want);
  const int64_t wave = int64_t(resident_ctas(kern, BLOCK, BYTES)) * sms;
  const int64_t resident = PERSIST ? wave : tiles;
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(tiles, resident)));
  a.prefetch_ahead = (PERSIST || (c.debug_flags & AK_DEBUG_NO_PREFETCH)) ? 0 : wave;
  if constexpr (CFG == CFG_RTS) {
    // one chunk of consecutive tiles per resident CTA: upsweep counts, then the
    // chunk-ordered pass (every CTA of the wave is resident, none waits on another)
    const int64_t want = std::max<int64_t>(1, std::min<int64_t>({tiles, wave, int64_t(RTS_MAX_CHUNKS)}));
    a.tiles_per_chunk = (tiles + want - 1) / want;
    const int64_t chunks = std::max<int64_t>(1, (tiles + a.tiles_per_chunk - 1) / a.tiles_per_chunk);
    a.chunk_cnt = c.chunk_cnt;
    a.debug_skip = 0;  // no look-back to starve
    for (int p = 0; p < PASSES; ++p) {
      a.pass = p;
      a.status_cur = nullptr;
      a.status_next = nullptr;
      if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p]), c.stream);
      chunk_hist_kernel<U, V, KIND, 512><<<unsigned(chunks), 512, 0, c.stream>>>(a, TILE);
      kern<<<unsigned(chunks), BLOCK, BYTES, c.stream>>>(a);
      if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p + 1]), c.stream);
    }
  } else
  for (int p = 0; p < PASSES; ++p) {
    a.pass = p;
    a.status_cur = c.status[p & 1];
    a.status_next = (p + 1 < PASSES) ? c.status[(p + 1) & 1] : nullptr;
    if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p]), c.stream);
    kern<<<grid, BLOCK, BYTES, c.stream>>>(a);
    if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p + 1]), c.stream);
  }
  {
    const int64_t want = (c.n + 1023) / 1024;
    const int g = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 4)));
    finish_kernel<U, V, HAS_V><<<g, 256, 0, c.stream>>>(a);
  }
  return cudaGetLastError();
}

// Sortperm of 8-byte keys in the default configuration with 32-bit look-back
// words: every pass launches the plain kernel and the packing one, and the
// passes of the upper key half also the kernel over packed words; the plan
// kernel says which format each pass has (onesweep.cuh: PassFormat) and only
// that variant runs, the others return at once.
template <typename U, int KIND>
cudaError_t run_passes_packed(const RadixCall &c, PassArgs<U, uint32_t> a) {
  using V = uint32_t;
  using P1 = PassKernel<U, V, true, KIND, uint32_t, CFG_DEFAULT>;   // key + index
  using P3 = PassKernel<U, V, false, KIND_UINT, uint32_t, CFG_DEFAULT>;  // packed words (tile shape)
  constexpr int BLOCK = P1::BLOCK;
  static_assert(P1::PERSIST && P3::BLOCK == BLOCK, "persistent default configuration");
  auto k1 = P1::kernel();
  auto k2 = onesweep_pass<U, V, true, KIND, uint32_t, BLOCK, P1::ITEMS, true, DIGIT_RADIX, false, FMT_PACK_OUT>;
  auto k3 = onesweep_pass<U, V, false, KIND_UINT, uint32_t, BLOCK, P3::ITEMS, true, DIGIT_RADIX, false, FMT_PACKED_IN>;
  cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, int(P1::BYTES));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(P1::BYTES));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k3, cudaFuncAttributeMaxDynamicSharedMemorySize, int(P3::BYTES));
  if (e != cudaSuccess) return e;
  constexpr int PASSES = sizeof(U);
  const int64_t tiles1 = (c.n + P1::TILE - 1) / P1::TILE;  // the larger count: its rows cover both shapes
  const int64_t tiles3 = (c.n + P3::TILE - 1) / P3::TILE;
  const int sms = device_sm_count();
  {
    constexpr int HB = 256;
    const int64_t want = (c.n + HB * 16 - 1) / (HB * 16);
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 8)));
    const int64_t zero_vec = tiles1 * RADIX * int64_t(sizeof(uint32_t)) / 16;
    hist_kernel<U, HB><<<grid, HB, 0, c.stream>>>(reinterpret_cast<const U *>(c.k_in), c.n, c.kind, a.flip,
                                                   c.counts, reinterpret_cast<uint4 *>(c.status[0]), zero_vec,
                                                   c.gate, c.gate_want);
  }
  plan_kernel<<<1, RADIX, 0, c.stream>>>(c.counts, c.n, PASSES, c.plan, c.hdr, c.path_tag, c.gate, c.gate_want,
                                         PASSES / 2);
  const unsigned g1 = unsigned(std::max<int64_t>(
      1, std::min<int64_t>(tiles1, int64_t(resident_ctas(k1, BLOCK, P1::BYTES)) * sms)));
  const unsigned g2 = unsigned(std::max<int64_t>(
      1, std::min<int64_t>(tiles1, int64_t(resident_ctas(k2, BLOCK, P1::BYTES)) * sms)));
  const unsigned g3 = unsigned(std::max<int64_t>(
      1, std::min<int64_t>(tiles3, int64_t(resident_ctas(k3, BLOCK, P3::BYTES)) * sms)));
  a.num_tiles = tiles1;
  a.prefetch_ahead = 0;
  a.fmt_check = 1;
  PassArgs<U, V> a3 = a;  // packed words: already transformed (no flip), unsigned digits
  a3.flip = U(0);
  a3.kind = KIND_UINT;
  a3.num_tiles = tiles3;
  for (int p = 0; p < PASSES; ++p) {
    a.pass = a3.pass = p;
    a.status_cur = a3.status_cur = c.status[p & 1];
    a.status_next = a3.status_next = (p + 1 < PASSES) ? c.status[(p + 1) & 1] : nullptr;
    if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p]), c.stream);
    k1<<<g1, BLOCK, P1::BYTES, c.stream>>>(a);
    k2<<<g2, BLOCK, P1::BYTES, c.stream>>>(a);
    if (p >= PASSES / 2) k3<<<g3, BLOCK, P3::BYTES, c.stream>>>(a3);
    if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p + 1]), c.stream);
  }
  {
    const int64_t want = (c.n + 1023) / 1024;
    const int g = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 4)));
    finish_kernel<U, V, true><<<g, 256, 0, c.stream>>>(a);
  }
  return cudaGetLastError();
}

template <typename U, typename V, bool HAS_V, int KIND>
cudaError_t run_status(const RadixCall &c) {
  PassArgs<U, V> a{};
  a.k_in = reinterpret_cast<const U *>(c.k_in);
  a.k_final = reinterpret_cast<U *>(c.k_final);
  a.k_alt0 = reinterpret_cast<U *>(c.k_alt0);
  a.k_alt1 = reinterpret_cast<U *>(c.k_alt1);
  a.v_in = reinterpret_cast<const V *>(c.v_in);
  a.v_final = reinterpret_cast<V *>(c.v_final);
  a.v_alt = reinterpret_cast<V *>(c.v_alt);
  a.n = c.n;
  a.kind = c.kind;
  a.flip = c.descending ? U(~U(0)) : U(0);
  a.mode = c.mode;
  a.plan = c.plan;
  a.hdr = c.hdr;
  a.timeout_ns = c.timeout_ns;
  a.debug_skip = (c.debug_flags & AK_DEBUG_SKIP_FIRST_TILE) ? 1 : 0;
  a.gate = c.gate;
  a.gate_want = c.gate_want;
  if constexpr (sizeof(U) == 16) {  // 128-bit keys: the default configuration only
    if constexpr (HAS_V && std::is_same<V, uint32_t>::value) {
      if (c.gather) {
        if (c.status_wide) return run_passes<U, V, HAS_V, KIND, unsigned long long, CFG_DEFAULT, DIGIT_GATHER>(c, a);
        return run_passes<U, V, HAS_V, KIND, uint32_t, CFG_DEFAULT, DIGIT_GATHER>(c, a);
      }
    }
    if (c.status_wide) return run_passes<U, V, HAS_V, KIND, unsigned long long, CFG_DEFAULT>(c, a);
    return run_passes<U, V, HAS_V, KIND, uint32_t, CFG_DEFAULT>(c, a);
  } else {
  if constexpr (HAS_V && std::is_same<V, uint32_t>::value && sizeof(U) == 8) {
    if (c.mode == MODE_PERM && !c.gather && !c.status_wide && c.tile_config == CFG_DEFAULT &&
        !(c.debug_flags & AK_DEBUG_NO_PACK))
      return run_passes_packed<U, KIND>(c, a);
  }
  if constexpr (HAS_V && std::is_same<V, uint32_t>::value) {
    if (c.gather) {  // low-memory sortperm: the shared-memory-staged configurations only
      if (c.status_wide) return run_passes<U, V, HAS_V, KIND, unsigned long long, 0, DIGIT_GATHER>(c, a);
      switch (c.tile_config) {
        case 1: return run_passes<U, V, HAS_V, KIND, uint32_t, 1, DIGIT_GATHER>(c, a);
        case 2: return run_passes<U, V, HAS_V, KIND, uint32_t, 2, DIGIT_GATHER>(c, a);
        default: return run_passes<U, V, HAS_V, KIND, uint32_t, 0, DIGIT_GATHER>(c, a);
      }
    }
  }
  if (c.status_wide) {  // 64-bit look-back words: configurations 0 and 3
    if (c.tile_config == CFG_WS) return run_passes<U, V, HAS_V, KIND, unsigned long long, CFG_WS>(c, a);
    return run_passes<U, V, HAS_V, KIND, unsigned long long, 0>(c, a);
  }
  switch (c.tile_config) {
    case 1: return run_passes<U, V, HAS_V, KIND, uint32_t, 1>(c, a);
    case 2: return run_passes<U, V, HAS_V, KIND, uint32_t, 2>(c, a);
    case CFG_WS: return run_passes<U, V, HAS_V, KIND, uint32_t, CFG_WS>(c, a);
    case CFG_RTS: return run_passes<U, V, HAS_V, KIND, uint32_t, CFG_RTS>(c, a);
    default: return run_passes<U, V, HAS_V, KIND, uint32_t, 0>(c, a);
  }
  }
}

template <typename U, int KIND>
cudaError_t radix_launch(const RadixCall &c) {
  if (c.n == 0) return cudaSuccess;
  if (c.mode == MODE_PERM) return run_status<U, uint32_t, true, KIND>(c);
  switch (c.val_bytes) {
    case 0: return run_status<U, uint32_t, false, KIND>(c);
    case 1: return run_status<U, uint8_t, true, KIND>(c);
    case 2: return run_status<U, uint16_t, true, KIND>(c);
    case 4: return run_status<U, uint32_t, true, KIND>(c);
    case 8: return run_status<U, unsigned long long, true, KIND>(c);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ak
