// radix_launch.cuh -- host launch sequence of the onesweep radix sort for one key width.
#pragma once

#include <algorithm>
#include <type_traits>

#include "internal.h"
#include "onesweep.cuh"

namespace ak {

// Tile shapes (threads per CTA, keys per thread) by key width and configuration.
template <typename U> struct TileShapes;
template <> struct TileShapes<uint16_t> {
  static constexpr int B[3] = {256, 256, 512};
  static constexpr int I[3] = {16, 8, 16};
};
template <> struct TileShapes<uint32_t> {
  static constexpr int B[3] = {256, 256, 512};
  static constexpr int I[3] = {15, 8, 12};
};
template <> struct TileShapes<uint64_t> {
  static constexpr int B[3] = {256, 256, 512};
  static constexpr int I[3] = {10, 6, 8};
};

template <typename U, typename V, bool HAS_V, typename S, int BLOCK, int ITEMS>
cudaError_t run_passes(const RadixCall &c, PassArgs<U, V> a) {
  using L = PassSmem<U, V, BLOCK, ITEMS, HAS_V>;
  auto kern = onesweep_pass<U, V, S, BLOCK, ITEMS, HAS_V>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L::BYTES));
  if (e != cudaSuccess) return e;
  const int64_t tiles = (c.n + L::TILE - 1) / L::TILE;
  a.num_tiles = tiles;
  constexpr int PASSES = sizeof(U);
  // histogram + zero the first pass's look-back words
  {
    constexpr int HB = 256;
    const int64_t want = (c.n + HB * 16 - 1) / (HB * 16);
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 8)));
    const int64_t zero_vec = tiles * RADIX * int64_t(sizeof(S)) / 16;
    hist_kernel<U, HB><<<grid, HB, 0, c.stream>>>(reinterpret_cast<const U *>(c.k_in), c.n, c.kind,
                                                   a.flip, c.counts,
                                                   reinterpret_cast<uint4 *>(c.status[0]), zero_vec);
  }
  plan_kernel<<<1, RADIX, 0, c.stream>>>(c.counts, c.n, PASSES, c.plan, c.hdr, c.path_tag);
  for (int p = 0; p < PASSES; ++p) {
    a.pass = p;
    a.status_cur = c.status[p & 1];
    a.status_next = (p + 1 < PASSES) ? c.status[(p + 1) & 1] : nullptr;
    if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p]), c.stream);
    kern<<<unsigned(tiles), BLOCK, L::BYTES, c.stream>>>(a);
    if (c.pass_events) cudaEventRecord(reinterpret_cast<cudaEvent_t>(c.pass_events[2 * p + 1]), c.stream);
  }
  {
    const int64_t want = (c.n + 1023) / 1024;
    const int grid = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 4)));
    finish_kernel<U, V, HAS_V><<<grid, 256, 0, c.stream>>>(a);
  }
  return cudaGetLastError();
}

template <typename U, typename V, bool HAS_V, typename S>
cudaError_t run_cfg(const RadixCall &c, const PassArgs<U, V> &a) {
  using T = TileShapes<U>;
  // values wider than 4 bytes and the 64-bit look-back words only take config 0
  const bool only0 = std::is_same<S, unsigned long long>::value || (HAS_V && sizeof(V) != 4);
  const int cfg = only0 ? 0 : c.tile_config;
  if constexpr (std::is_same<S, unsigned long long>::value || (HAS_V && sizeof(V) != 4)) {
    return run_passes<U, V, HAS_V, S, T::B[0], T::I[0]>(c, a);
  } else {
    switch (cfg) {
      case 1: return run_passes<U, V, HAS_V, S, T::B[1], T::I[1]>(c, a);
      case 2: return run_passes<U, V, HAS_V, S, T::B[2], T::I[2]>(c, a);
      default: return run_passes<U, V, HAS_V, S, T::B[0], T::I[0]>(c, a);
    }
  }
}

template <typename U, typename V, bool HAS_V>
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
  if (c.status_wide) return run_cfg<U, V, HAS_V, unsigned long long>(c, a);
  return run_cfg<U, V, HAS_V, uint32_t>(c, a);
}

template <typename U>
cudaError_t radix_launch(const RadixCall &c) {
  if (c.n == 0) return cudaSuccess;
  if (c.mode == MODE_PERM) return run_status<U, uint32_t, true>(c);
  switch (c.val_bytes) {
    case 0: return run_status<U, uint32_t, false>(c);
    case 1: return run_status<U, uint8_t, true>(c);
    case 2: return run_status<U, uint16_t, true>(c);
    case 4: return run_status<U, uint32_t, true>(c);
    case 8: return run_status<U, unsigned long long, true>(c);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ak
