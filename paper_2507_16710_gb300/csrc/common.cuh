// common.cuh -- device helpers shared by every kernel of the sort library.
//
//  * the order-preserving key transform (Julia isless -> unsigned radix key)
//  * the device status word and bounded waits
//  * thin inline-PTX wrappers for mbarrier + cp.async.bulk (the sm_90+/sm_103a
//    bulk-copy engine used to stage whole tiles into shared memory)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/ak_sort.h"

namespace ak {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int MAX_PASSES = 16;  // 128-bit keys

// KIND_FLOAT: IEEE binary16/32/64 by the key width; KIND_BF16: bfloat16 (the
// upper half of a binary32: 8 exponent bits), 16-bit keys only.
enum KeyKind : int { KIND_UINT = 0, KIND_SINT = 1, KIND_FLOAT = 2, KIND_BF16 = 3 };

// ----------------------------------------------------------------- key transform
// Julia isless on the raw bits of a key, as an unsigned integer order:
//   unsigned ints: identity; signed ints: flip the sign bit;
//   floats: NaN (any sign/payload) -> all ones (after +Inf, all NaNs tie);
//           negative -> all bits flipped (so -0.0 = ~0x80.. sits just below
//           +0.0 = 0x80..); non-negative -> sign bit flipped.
// Descending (Julia rev=true) complements the result; ties keep input order
// because every pass is stable.  Only the digits are derived from this value:
// the data moved is always the raw key bits.
template <typename U> struct FloatBits;
template <> struct FloatBits<uint16_t> { static constexpr uint16_t EXP = 0x7C00u; };
template <> struct FloatBits<uint32_t> { static constexpr uint32_t EXP = 0x7F800000u; };
template <> struct FloatBits<uint64_t> { static constexpr uint64_t EXP = 0x7FF0000000000000ull; };

// Exponent field of a float kind (all ones: infinity, above it: NaN).
template <int KIND, typename U>
__host__ __device__ constexpr U float_exp() {
  return KIND == KIND_BF16 ? U(0x7F80u) : FloatBits<U>::EXP;
}
constexpr bool is_float_kind(int kind) { return kind == KIND_FLOAT || kind == KIND_BF16; }

template <typename U>
__device__ __forceinline__ U radix_key(U u, int kind, U flip) {
  constexpr U SIGN = U(U(1) << (8 * sizeof(U) - 1));
  U r;
  if constexpr (sizeof(U) > 8) {  // 128-bit keys are integers
    r = kind == KIND_SINT ? U(u ^ SIGN) : u;
  } else if (is_float_kind(kind)) {
    const U mag = U(u & U(~SIGN));
    r = (u & SIGN) ? U(~u) : U(u ^ SIGN);
    if (mag > (kind == KIND_BF16 ? float_exp<KIND_BF16, U>() : FloatBits<U>::EXP)) r = U(~U(0));
  } else if (kind == KIND_SINT) {
    r = U(u ^ SIGN);
  } else {
    r = u;
  }
  return U(r ^ flip);
}

// Same transform with the key kind fixed at compile time (no per-key branches).
template <int KIND, typename U>
__device__ __forceinline__ U radix_key_t(U u, U flip) {
  constexpr U SIGN = U(U(1) << (8 * sizeof(U) - 1));
  if constexpr (KIND == KIND_FLOAT || KIND == KIND_BF16) {
    // negative -> ~u, non-negative -> u ^ SIGN: xor with (arithmetic sign mask | SIGN)
    using S = typename std::make_signed<U>::type;
    const U neg = U(S(u) >> (8 * sizeof(U) - 1));
    U r = U(u ^ (neg | SIGN));
    r = (U(u & U(~SIGN)) > float_exp<KIND, U>()) ? U(~U(0)) : r;
    return U(r ^ flip);
  } else if constexpr (KIND == KIND_SINT) {
    return U(u ^ SIGN ^ flip);
  } else {
    return U(u ^ flip);
  }
}

template <typename U>
__device__ __forceinline__ uint32_t digit_of(U r, int shift) {
  if constexpr (sizeof(U) > 8)  // the 32-bit word that holds the digit
    return (uint32_t(r >> (shift & ~31)) >> (shift & 31)) & (RADIX - 1);
  else
    return uint32_t(r >> shift) & (RADIX - 1);
}

using u128 = unsigned __int128;

// ----------------------------------------------------------------- status word
// Header at offset 0 of every workspace.  `status` holds the first device-side
// error (ak_status); kernels never trap.
struct DevHeader {
  uint32_t status;
  uint32_t pad0;
  uint32_t tile_counter[16];   // dynamic tile ids, one per digit pass
  uint32_t work_counter[8];    // work queues of the persistent kernels
  ak_info info;
};

__device__ __forceinline__ void set_error(DevHeader *h, uint32_t code) {
  atomicCAS(&h->status, 0u, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// --------------------------------------------------------- mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Non-blocking probe of phase `parity`; true once the phase has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bulk copy global -> shared of `bytes` (multiple of 16, both addresses 16-byte
// aligned), completing on `bar` with transaction bytes.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Hint: pull `bytes` (multiple of 16, 16-byte aligned) of global memory into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src_gmem, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src_gmem), "r"(bytes) : "memory");
}

// Bounded wait on an mbarrier phase.  On timeout the error is recorded and the
// caller must not touch the destination buffer until a second bounded wait
// confirms the copy landed (see wait_copy_or_fail).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 15u) == 0 && globaltimer_ns() - t0 > timeout_ns) return false;
  }
  return true;
}

// Named barriers: a subset of the CTA's warps synchronises (bar.sync) or only
// signals its arrival (bar.arrive); `nthreads` counts every participant.
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_arrive(uint32_t id, uint32_t nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ------------------------------------------------------------------ warp utils
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan over a CTA of NT threads (NT multiple of 32); `scratch` holds
// NT/32 + 1 values.  Returns the exclusive prefix; *total gets the CTA sum.
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *scratch, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = warp_inclusive_scan(v);
  if (lane == 31) scratch[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < NT / 32) ? scratch[lane] : T(0);
    T wi = warp_inclusive_scan(w);
    if (lane < NT / 32) scratch[lane] = wi - w;
    if (lane == NT / 32 - 1) scratch[NT / 32] = wi;
  }
  __syncthreads();
  T out = scratch[warp] + inc - v;
  *total = scratch[NT / 32];
  __syncthreads();
  return out;
}

}  // namespace ak
