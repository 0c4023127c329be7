// seg_launch.cuh -- host launch of the segmented sort for one key word width and kind.
#pragma once

#include <algorithm>
#include <utility>

#include "internal.h"
#include "merge.cuh"
#include "radix_launch.cuh"
#include "segsort.cuh"
#include "segsplit.cuh"

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
  // without offsets: one segment, or (merge) tiles of the shared-memory capacity
  a.tile_len = c.off ? 0 : (c.merge ? int64_t(CAP) : c.n);
  a.nseg = c.off ? c.nseg : (c.n + a.tile_len - 1) / a.tile_len;
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
  const int sms = device_sm_count();
  const bool split = c.off && c.nseg > 0 && c.split_state;
  if (split) {  // long segments cut into buckets by all CTAs first (segsplit.cuh)
    constexpr int SI = split_items(sizeof(U), HAS_V ? sizeof(V) : 0);
    constexpr int64_t T = SPLIT_BLOCK * SI;
    using SL = SplitSmem<U, V, HAS_V, KIND, SI>;
    auto st = reinterpret_cast<SplitState *>(c.split_state);
    auto big = reinterpret_cast<BigSeg *>(c.split_big);
    auto bk = reinterpret_cast<BucketItem *>(c.split_buckets);
    const int64_t g = (c.nseg + 255) / 256;
    const int64_t split_min = c.split_min > 0 ? c.split_min : (c.split_min < 0 ? INT64_MAX : int64_t(SPLIT_MIN_CAPS) * CAP);
    split_classify_kernel<<<unsigned(g), 256, 0, c.stream>>>(c.off, c.nseg, c.n, CAP, split_min, c.order, big, st,
                                                             c.gate, c.gate_want);
    split_tiles_kernel<<<1, 1024, 0, c.stream>>>(big, st, T, c.gate, c.gate_want);
    split_vary_kernel<U, KIND><<<unsigned(sms * 4), SPLIT_BLOCK, 0, c.stream>>>(a.keys, big, st, T, a.flip, c.gate,
                                                                                c.gate_want);
    split_count_kernel<U, KIND><<<unsigned(sms * 4), SPLIT_BLOCK, 0, c.stream>>>(a.keys, big, st, T, CAP, a.flip,
                                                                                 c.split_tcount, c.gate, c.gate_want);
    split_scan_kernel<<<unsigned(sms * 8), RADIX, 0, c.stream>>>(big, st, c.split_tcount, bk, c.gate, c.gate_want);
    auto sk = split_scatter_kernel<U, V, HAS_V, KIND, SI>;
    e = cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SL::BYTES));
    if (e != cudaSuccess) return e;
    const int64_t sres = int64_t(resident_ctas(sk, SPLIT_BLOCK, SL::BYTES)) * sms;
    sk<<<unsigned(sres), SPLIT_BLOCK, SL::BYTES, c.stream>>>(a.keys, a.vals, a.alt_k, a.alt_v, big, st,
                                                               c.split_tcount, CAP, a.flip, c.gate, c.gate_want);
    a.split = st;
    a.buckets = bk;
  } else if (c.off && c.nseg > 0) {
    const int64_t g = (c.nseg + 255) / 256;
    classify_kernel<<<unsigned(g), 256, 0, c.stream>>>(c.off, c.nseg, c.n, CAP, c.order, c.counters, c.gate,
                                                       c.gate_want);
  }
  const int64_t resident = int64_t(resident_ctas(kern, SEG_BLOCK, Lay::BYTES)) * sms;
  // with the split the work items (buckets + short segments) are counted on the device
  const unsigned grid = unsigned(std::max<int64_t>(1, split ? resident : std::min<int64_t>(a.nseg, resident)));
  kern<<<grid, SEG_BLOCK, Lay::BYTES, c.stream>>>(a);
  if (!c.off && c.merge && c.n > CAP) {
    // merge rounds: runs of CAP * 2^r, ping-pong between the keys and the workspace copy
    constexpr int MB = 256, MI = 8, MCH = MB * MI;
    auto mk = merge_pass_kernel<U, V, HAS_V, KIND, MB, MI>;
    const int64_t mres = int64_t(resident_ctas(mk, MB, 0)) * device_sm_count();
    U *src_k = a.keys, *dst_k = a.alt_k;
    V *src_v = a.vals, *dst_v = a.alt_v;
    for (int64_t w = CAP; w < c.n; w *= 2) {
      const int64_t pairs = (c.n + 2 * w - 1) / (2 * w);
      const int64_t cpp = (2 * w + MCH - 1) / MCH;
      const int64_t chunks = pairs * cpp;
      const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(chunks, mres)));
      mk<<<g, MB, 0, c.stream>>>(src_k, src_v, dst_k, dst_v, c.n, w, a.flip, cpp, chunks);
      std::swap(src_k, dst_k);
      std::swap(src_v, dst_v);
    }
    if (src_k != a.keys) {  // an odd number of rounds: the result is in the workspace copy
      e = cudaMemcpyAsync(a.keys, src_k, size_t(c.n) * sizeof(U), cudaMemcpyDeviceToDevice, c.stream);
      if (e == cudaSuccess && HAS_V)
        e = cudaMemcpyAsync(a.vals, src_v, size_t(c.n) * sizeof(V), cudaMemcpyDeviceToDevice, c.stream);
      if (e != cudaSuccess) return e;
    }
  }
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
