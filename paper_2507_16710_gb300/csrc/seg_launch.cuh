// seg_launch.cuh -- host launch of the segmented sort for one key word width and kind.
#pragma once

#include <algorithm>

#include "internal.h"
#include "radix_launch.cuh"
#include "segsort.cuh"

namespace ak {

constexpr int SEG_BLOCK = 512;
// keys ranked per thread and chunk: at most 8, and a chunk never exceeds CAP
constexpr int seg_items(int key_bytes, int val_bytes) {
  return seg_cap(key_bytes, val_bytes) / SEG_BLOCK < 8 ? seg_cap(key_bytes, val_bytes) / SEG_BLOCK : 8;
}

template <typename U, typename V, bool HAS_V, int KIND>
cudaError_t seg_run(const SegCall &c) {
  constexpr int CAP = seg_cap(sizeof(U), HAS_V ? sizeof(V) : 0);
  constexpr int ITEMS = seg_items(sizeof(U), HAS_V ? sizeof(V) : 0);
  using Lay = SegSmem<U, V, HAS_V, KIND, SEG_BLOCK, ITEMS, CAP>;
  auto kern = segsort_kernel<U, V, HAS_V, KIND, SEG_BLOCK, ITEMS, CAP>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Lay::BYTES));
  if (e != cudaSuccess) return e;
  SegArgs<U, V> a{};
  a.off = c.off;
  a.nseg = c.off ? c.nseg : 1;
  a.n = c.n;
  a.order = c.off ? c.order : nullptr;
  a.hdr = c.hdr;
  a.path_tag = c.path_tag;
  a.gate = c.gate;
  a.gate_want = c.gate_want;
  a.keys = reinterpret_cast<U *>(c.keys);
  a.vals = reinterpret_cast<V *>(c.vals);
  a.alt_k = reinterpret_cast<U *>(c.alt_k);
  a.alt_v = reinterpret_cast<V *>(c.alt_v);
  a.flip = c.descending ? U(~U(0)) : U(0);
  a.seg_base = 0;
  if (c.off && c.nseg > 0) {
    const int64_t g = (c.nseg + 255) / 256;
    classify_kernel<<<unsigned(g), 256, 0, c.stream>>>(c.off, c.nseg, c.n, CAP, c.order, c.counters, c.gate,
                                                       c.gate_want);
  }
  const int64_t resident = int64_t(resident_ctas(kern, SEG_BLOCK, Lay::BYTES)) * device_sm_count();
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(a.nseg, resident)));
  kern<<<grid, SEG_BLOCK, Lay::BYTES, c.stream>>>(a);
  return cudaGetLastError();
}

template <typename U, int KIND>
cudaError_t seg_launch(const SegCall &c) {
  if (c.n == 0 || (c.off && c.nseg == 0)) return cudaSuccess;
  switch (c.val_bytes) {
    case 0: return seg_run<U, uint32_t, false, KIND>(c);
    case 1: return seg_run<U, uint8_t, true, KIND>(c);
    case 2: return seg_run<U, uint16_t, true, KIND>(c);
    case 4: return seg_run<U, uint32_t, true, KIND>(c);
    case 8: return seg_run<U, unsigned long long, true, KIND>(c);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ak
