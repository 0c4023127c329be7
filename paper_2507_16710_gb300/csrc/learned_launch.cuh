// learned_launch.cuh -- launch sequence of the learned-CDF bucketing path for one
// key word width and key kind.
//
//   sample -> x-hat -> sort the sample (the library's radix path) -> knot counts
//   -> train the residual MLP -> monotone table -> bucket histogram -> plan
//   -> 1-2 stable onesweep passes on the bucket-id bytes -> per-bucket sort
//   (the segmented sort, one segment per bucket)
// The device decides whether the buckets are usable: already on the sample
// (lm_choose_kernel: more than a quarter of the sample in windows the model
// would overload far beyond capacity) or on the full bucket histogram
// (lm_plan_kernel: more than a quarter of the keys in buckets above 16 times
// the shared-memory capacity).  Either sets use_plain; every learned kernel
// after it returns at once and the plain radix sequence (launched after them,
// gated the other way) sorts instead.  No
// host synchronisation, so the whole call can be captured in a CUDA graph.
#pragma once

#include <algorithm>
#include <cstddef>

#include "internal.h"
#include "learned.cuh"
#include "radix_launch.cuh"

namespace ak {

// Full histogram of bucket ids: 16-bit shared counters (two per word); a
// counter that reaches 0x8000 moves 0x8000 to the global count, so no counter
// can carry into its neighbour while up to 1024 threads increment it.  With
// `ids`, every key's bucket id is also stored (the passes then carry it as a
// value instead of evaluating the model again).
template <typename U, int KIND>
__global__ void __launch_bounds__(1024) lm_hist_kernel(const U *__restrict__ keys, int64_t n, U flip,
                                                       const LearnedModel *md, uint32_t *counts, uint4 *zero_buf,
                                                       int64_t zero_vec, uint16_t *ids) {
  if (md->use_plain) return;
  extern __shared__ uint32_t hw[];
  const uint32_t nb = md->nbuckets;
  for (uint32_t i = threadIdx.x; i < nb / 2; i += blockDim.x) hw[i] = 0u;
  const int64_t gtid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = gtid; i < zero_vec; i += stride) zero_buf[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int64_t i = gtid; i < n; i += stride) {
    const uint32_t b = lm_key_bucket<KIND>(md, keys[i], flip);
    if (ids) ids[i] = uint16_t(b);
    const uint32_t sh = (b & 1u) * 16u;
    const uint32_t old = atomicAdd(&hw[b >> 1], 1u << sh);
    if (((old >> sh) & 0xFFFFu) == 0x7FFFu) {
      atomicSub(&hw[b >> 1], 0x8000u << sh);
      atomicAdd(&counts[b], 0x8000u);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
    const uint32_t c = (hw[i >> 1] >> ((i & 1u) * 16u)) & 0xFFFFu;
    if (c) atomicAdd(&counts[i], c);
  }
}

// Plan of the learned passes, CSR offsets of the buckets, statistics and the
// fallback decision.  One CTA of 1024 threads.
__global__ void lm_plan_kernel(const uint32_t *counts, int64_t n, LearnedModel *md, RadixPlan *plan, DevHeader *hdr,
                               int64_t *seg_off, int64_t cap);

template <typename U, int KIND>
cudaError_t radix_launch_kind(const RadixCall &c);
template <> inline cudaError_t radix_launch_kind<uint16_t, KIND_UINT>(const RadixCall &c) { return radix_launch_u16_uint(c); }
template <> inline cudaError_t radix_launch_kind<uint16_t, KIND_SINT>(const RadixCall &c) { return radix_launch_u16_sint(c); }
template <> inline cudaError_t radix_launch_kind<uint16_t, KIND_FLOAT>(const RadixCall &c) { return radix_launch_u16_float(c); }
template <> inline cudaError_t radix_launch_kind<uint16_t, KIND_BF16>(const RadixCall &c) { return radix_launch_u16_bf16(c); }
template <> inline cudaError_t radix_launch_kind<uint32_t, KIND_UINT>(const RadixCall &c) { return radix_launch_u32_uint(c); }
template <> inline cudaError_t radix_launch_kind<uint32_t, KIND_SINT>(const RadixCall &c) { return radix_launch_u32_sint(c); }
template <> inline cudaError_t radix_launch_kind<uint32_t, KIND_FLOAT>(const RadixCall &c) { return radix_launch_u32_float(c); }
template <> inline cudaError_t radix_launch_kind<uint64_t, KIND_UINT>(const RadixCall &c) { return radix_launch_u64_uint(c); }
template <> inline cudaError_t radix_launch_kind<uint64_t, KIND_SINT>(const RadixCall &c) { return radix_launch_u64_sint(c); }
template <> inline cudaError_t radix_launch_kind<uint64_t, KIND_FLOAT>(const RadixCall &c) { return radix_launch_u64_float(c); }

template <typename U, int KIND>
cudaError_t seg_launch_kind(const SegCall &c);
template <> inline cudaError_t seg_launch_kind<uint16_t, KIND_UINT>(const SegCall &c) { return seg_launch_u16_uint(c); }
template <> inline cudaError_t seg_launch_kind<uint16_t, KIND_SINT>(const SegCall &c) { return seg_launch_u16_sint(c); }
template <> inline cudaError_t seg_launch_kind<uint16_t, KIND_FLOAT>(const SegCall &c) { return seg_launch_u16_float(c); }
template <> inline cudaError_t seg_launch_kind<uint16_t, KIND_BF16>(const SegCall &c) { return seg_launch_u16_bf16(c); }
template <> inline cudaError_t seg_launch_kind<uint32_t, KIND_UINT>(const SegCall &c) { return seg_launch_u32_uint(c); }
template <> inline cudaError_t seg_launch_kind<uint32_t, KIND_SINT>(const SegCall &c) { return seg_launch_u32_sint(c); }
template <> inline cudaError_t seg_launch_kind<uint32_t, KIND_FLOAT>(const SegCall &c) { return seg_launch_u32_float(c); }
template <> inline cudaError_t seg_launch_kind<uint64_t, KIND_UINT>(const SegCall &c) { return seg_launch_u64_uint(c); }
template <> inline cudaError_t seg_launch_kind<uint64_t, KIND_SINT>(const SegCall &c) { return seg_launch_u64_sint(c); }
template <> inline cudaError_t seg_launch_kind<uint64_t, KIND_FLOAT>(const SegCall &c) { return seg_launch_u64_float(c); }

// The learned passes (digits = bytes of the bucket id) with the radix pass
// kernel.  DIGIT_LEARNED evaluates the model for every key in every pass;
// DIGIT_VALUE (keys-only sorts) carries the id the histogram stored as a
// 16-bit value instead: two extra bytes read and written per key and pass in
// place of the model evaluation.
template <typename U, typename V, bool HAS_V, int KIND, typename S, int DIGIT = DIGIT_LEARNED>
cudaError_t lm_passes(const RadixCall &c, const LearnedCall &lc) {
  constexpr int CFG = CFG_DEFAULT;
  using P = PassKernel<U, V, HAS_V, KIND, S, CFG, DIGIT>;
  constexpr int BLOCK = P::BLOCK;
  constexpr bool PERSIST = P::PERSIST;
  constexpr int TILE = P::TILE;
  constexpr size_t BYTES = P::BYTES;
  auto kern = P::kernel();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(BYTES));
  if (e != cudaSuccess) return e;
  const int64_t tiles = (c.n + TILE - 1) / TILE;
  PassArgs<U, V> a{};
  a.k_in = reinterpret_cast<const U *>(c.k_in);
  a.k_final = reinterpret_cast<U *>(c.k_final);
  a.k_alt0 = reinterpret_cast<U *>(c.k_alt0);
  a.k_alt1 = reinterpret_cast<U *>(c.k_alt1);
  if constexpr (DIGIT == DIGIT_VALUE) {  // ids: histogram -> pass 1 -> pass 2 (-> the first array again)
    a.v_in = reinterpret_cast<const V *>(lc.ids);
    a.v_final = reinterpret_cast<V *>(lc.ids);
    a.v_alt = reinterpret_cast<V *>(lc.ids_alt);
  } else {
    a.v_in = reinterpret_cast<const V *>(c.v_in);
    a.v_final = reinterpret_cast<V *>(c.v_final);
    a.v_alt = reinterpret_cast<V *>(c.v_alt);
  }
  a.n = c.n;
  a.kind = c.kind;
  a.flip = c.descending ? U(~U(0)) : U(0);
  a.mode = MODE_INPLACE;
  a.plan = c.plan;
  a.hdr = c.hdr;
  a.timeout_ns = c.timeout_ns;
  a.num_tiles = tiles;
  a.model = lc.model;
  a.gate = &lc.model->use_plain;
  a.gate_want = 0;
  // histogram of bucket ids (zeroes the first pass's look-back words)
  {
    const int64_t zero_vec = tiles * RADIX * int64_t(sizeof(S)) / 16;
    const size_t hsm = size_t(lc.nbuckets / 2) * 4;
    auto hk = lm_hist_kernel<U, KIND>;
    e = cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, int(hsm));
    if (e != cudaSuccess) return e;
    hk<<<device_sm_count(), 1024, hsm, c.stream>>>(reinterpret_cast<const U *>(c.k_in), c.n, a.flip, lc.model,
                                                   lc.bucket_counts, reinterpret_cast<uint4 *>(c.status[0]),
                                                   zero_vec, DIGIT == DIGIT_VALUE ? lc.ids : nullptr);
  }
  lm_plan_kernel<<<1, 1024, 0, c.stream>>>(lc.bucket_counts, c.n, lc.model, c.plan, c.hdr, lc.seg_off, lc.seg_capacity);
  const int passes = int((lc.bucket_bits + RADIX_BITS - 1) / RADIX_BITS);
  const int64_t wave = int64_t(resident_ctas(kern, BLOCK, BYTES)) * device_sm_count();
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(tiles, PERSIST ? wave : tiles)));
  a.prefetch_ahead = PERSIST ? 0 : wave;
  for (int p = 0; p < passes; ++p) {
    a.pass = p;
    a.status_cur = c.status[p & 1];
    a.status_next = (p + 1 < passes) ? c.status[(p + 1) & 1] : nullptr;
    kern<<<grid, BLOCK, BYTES, c.stream>>>(a);
  }
  {
    const int64_t want = (c.n + 1023) / 1024;
    const int g = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 4)));
    finish_kernel<U, V, HAS_V><<<g, 256, 0, c.stream>>>(a);
  }
  return cudaGetLastError();
}

template <typename U, typename V, bool HAS_V, int KIND>
cudaError_t lm_passes_s(const RadixCall &c, const LearnedCall &lc) {
  if (!HAS_V && lc.ids && lc.ids_alt) {  // keys only: carry the bucket id as a 16-bit value
    if (c.status_wide) return lm_passes<U, uint16_t, true, KIND, unsigned long long, DIGIT_VALUE>(c, lc);
    return lm_passes<U, uint16_t, true, KIND, uint32_t, DIGIT_VALUE>(c, lc);
  }
  if (c.status_wide) return lm_passes<U, V, HAS_V, KIND, unsigned long long>(c, lc);
  return lm_passes<U, V, HAS_V, KIND, uint32_t>(c, lc);
}

template <typename U, int KIND>
cudaError_t learned_launch(const RadixCall &c, const LearnedCall &lc) {
  if (c.n == 0) return cudaSuccess;
  cudaError_t e;
  const U flip = c.descending ? U(~U(0)) : U(0);
  const int sms = device_sm_count();
  // 1. sample (radix keys) and its range; 2. sort it by radix key
  const int g = int(std::min<int64_t>((lc.m + 255) / 256, int64_t(sms) * 4));
  lm_sample_kernel<U, KIND><<<g, 256, 0, c.stream>>>(reinterpret_cast<const U *>(c.k_in), c.n, flip, lc.m, lc.seed,
                                                     lc.sample_r, lc.model, nullptr);
  if ((e = radix_launch_u64_uint(lc.sample_sort)) != cudaSuccess) return e;
  // 3. x-hat of the sorted sample in each coordinate, the knots of each, the
  //    coordinate whose piecewise-linear fit is closer; residual MLP; table
  constexpr int VBYTES = (KIND == KIND_FLOAT && sizeof(U) >= 4) ? int(sizeof(U)) : 0;
  lm_xhat_kernel<<<g, 256, 0, c.stream>>>(lc.sample_r, lc.m, lc.model, lc.xs, VBYTES ? lc.xs_v : nullptr, VBYTES,
                                          (unsigned long long)flip, nullptr);
  lm_knots_kernel<<<1, LM_KNOTS, 0, c.stream>>>(lc.xs, lc.m, nullptr, lc.model, nullptr);
  if (VBYTES) {
    float *cv = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(lc.model) + offsetof(LearnedModel, c_v));
    lm_knots_kernel<<<1, LM_KNOTS, 0, c.stream>>>(lc.xs_v, lc.m, cv, nullptr, nullptr);
  }
  lm_fit_error_kernel<<<g, 256, 0, c.stream>>>(lc.xs, VBYTES ? lc.xs_v : nullptr, lc.m, lc.model, nullptr);
  lm_choose_kernel<<<1, LM_KNOTS, 0, c.stream>>>(lc.model, VBYTES ? 1 : 0, c.hdr, c.n, lc.nbuckets, nullptr);
  const uint32_t *fallback = &lc.model->use_plain;  // every later learned kernel skips itself once set
  if (lc.train_steps > 0) {
    const int smem = int(sizeof(GradSmem));
    if ((e = cudaFuncSetAttribute(lm_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(LM_TRAIN_CTAS);
    cfg.blockDim = dim3(LM_TRAIN_BLOCK);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // all CTAs co-resident for the grid barrier
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if ((e = cudaLaunchKernelEx(&cfg, lm_train_kernel, static_cast<const float *>(lc.xs),
                                static_cast<const float *>(VBYTES ? lc.xs_v : nullptr), lc.m, lc.model, lc.partials,
                                lc.train_steps, lc.lr, lc.seed ^ 0x5EEDu, c.hdr, c.timeout_ns, fallback)) !=
        cudaSuccess)
      return e;
  }
  // the bucket table: the piecewise-linear CDF alone, or with the trained
  // residual when that gives the sorted sample a strictly smaller largest
  // bucket (the loss is a mean; the sort pays for the largest bucket)
  const float *xs_v = VBYTES ? lc.xs_v : nullptr;
  const int rg = int(std::min<int64_t>((lc.m + 255) / 256, int64_t(sms) * 8));
  lm_table_kernel<<<1, 1024, 0, c.stream>>>(lc.model, 0, lc.nbuckets, lc.bucket_bits, fallback);
  lm_sample_runs_kernel<<<rg, 256, 0, c.stream>>>(lc.xs, xs_v, lc.m, lc.model, 0, fallback);
  if (lc.train_steps > 0) {
    lm_table_kernel<<<1, 1024, 0, c.stream>>>(lc.model, 1, lc.nbuckets, lc.bucket_bits, fallback);
    lm_sample_runs_kernel<<<rg, 256, 0, c.stream>>>(lc.xs, xs_v, lc.m, lc.model, 1, fallback);
  }
  lm_pick_kernel<<<1, 1, 0, c.stream>>>(lc.model, c.hdr, fallback);
  if (lc.train_steps > 0)  // the table of the choice (the PL one was overwritten)
    lm_table_kernel<<<1, 1024, 0, c.stream>>>(lc.model, 2, lc.nbuckets, lc.bucket_bits, fallback);
  // 4. bucket histogram, plan, learned passes (all skip themselves on fallback)
  switch (c.val_bytes) {
    case 0: e = lm_passes_s<U, uint32_t, false, KIND>(c, lc); break;
    case 1: e = lm_passes_s<U, uint8_t, true, KIND>(c, lc); break;
    case 2: e = lm_passes_s<U, uint16_t, true, KIND>(c, lc); break;
    case 4: e = lm_passes_s<U, uint32_t, true, KIND>(c, lc); break;
    case 8: e = lm_passes_s<U, unsigned long long, true, KIND>(c, lc); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  // 5. sort inside every bucket
  if ((e = seg_launch_kind<U, KIND>(lc.finish)) != cudaSuccess) return e;
  // 6. fallback: the plain radix sequence, run only when use_plain was set
  RadixCall plain = c;
  plain.gate = &lc.model->use_plain;
  plain.gate_want = 1;
  plain.path_tag = 0;
  return radix_launch_kind<U, KIND>(plain);
}

}  // namespace ak
