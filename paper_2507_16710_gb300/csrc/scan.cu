// scan.cu -- accumulate: single-pass prefix scan with decoupled look-back
// (Sec. II-B, accumulate, inclusive and exclusive, with opportunistic
// look-back after Merrill and Garland, "Single-pass Parallel Prefix Scan with
// Decoupled Look-back", 2016).
//
// out[i] = init (+) x[0] (+) ... (+) x[i]      (inclusive)
// out[i] = init (+) x[0] (+) ... (+) x[i - 1]  (exclusive, out[0] = init)
// for (+) = + (integers wrap in their width), Julia max, Julia min.
//
// HBM bound: n * w bytes read and n * w written.  Design for GB300:
//  * persistent CTAs (resident count) take 32 KB tiles from an atomic counter,
//    in increasing order, so a tile only ever waits on tiles already held by
//    running CTAs -- forward progress needs no co-residency; a CTA claims its
//    next tile as soon as the current one's aggregate is published and loads
//    it into registers while warp 0 looks back;
//  * each thread loads 64 contiguous bytes (32 for 16-bit keys: four or two
//    16-byte vector loads when the tile is whole and the pointers 16-byte
//    aligned) and scans them in registers; the CTA scans the 512 thread
//    totals with warp shuffles;
//  * the tile publishes its aggregate, then warp 0 looks back over up to 32
//    predecessors at a time, stops at the nearest inclusive prefix and
//    publishes its own inclusive prefix;
//  * status: a 32-bit flag (release store / acquire load, gpu scope) beside
//    two write-once 64-bit slots, the aggregate and the inclusive prefix, so a
//    reader that saw one flag value can never pick up the other slot's value
//    (one scheme for every key width);
//  * every wait is bounded by the globaltimer: on expiry the CTA records
//    AK_ERR_TIMEOUT, takes the identity for the missing prefix and finishes.
//
// Identities (x (+) e == x bit for bit, -0.0 and NaN included): + on floats
// -0.0, on integers 0; max -Inf or the lowest integer; min +Inf or the highest.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <limits>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace ak {

constexpr int SCAN_BLOCK = 512;
// 16-byte vectors per thread: 64 bytes (32 bytes for 16-bit keys, whose values
// each take a register)
constexpr int scan_vecs(int key_bytes) { return key_bytes == 2 ? 2 : 4; }
constexpr int scan_tile(int key_bytes) { return SCAN_BLOCK * scan_vecs(key_bytes) * 16 / key_bytes; }
constexpr uint32_t SCAN_FLAG_AGG = 1, SCAN_FLAG_INC = 2;

// ----------------------------------------------------------------- operators
template <typename T, int OP> struct ScanOp;

// + : integers in unsigned arithmetic (wraps, no signed overflow), floats IEEE
template <typename T> struct ScanOp<T, AK_SCAN_ADD> {
  static __device__ __forceinline__ T identity() {
    if constexpr (std::is_floating_point<T>::value) return T(-0.0);
    else return T(0);
  }
  static __device__ __forceinline__ T apply(T a, T b) {
    if constexpr (std::is_floating_point<T>::value) {
      return a + b;
    } else {
      using UT = typename std::make_unsigned<T>::type;
      return T(UT(UT(a) + UT(b)));
    }
  }
};

// Julia max: a NaN operand wins; +0.0 above -0.0
template <typename T> struct ScanOp<T, AK_SCAN_MAX> {
  static __device__ __forceinline__ T identity() {
    if constexpr (std::is_floating_point<T>::value) return -std::numeric_limits<T>::infinity();
    else return std::numeric_limits<T>::lowest();
  }
  static __device__ __forceinline__ T apply(T a, T b) {
    if constexpr (std::is_floating_point<T>::value) {
      if (a != a) return a;
      if (b != b) return b;
      if (a == b) return signbit(a) ? b : a;
      return a > b ? a : b;
    } else {
      return a > b ? a : b;
    }
  }
};

// Julia min: a NaN operand wins; -0.0 below +0.0
template <typename T> struct ScanOp<T, AK_SCAN_MIN> {
  static __device__ __forceinline__ T identity() {
    if constexpr (std::is_floating_point<T>::value) return std::numeric_limits<T>::infinity();
    else return std::numeric_limits<T>::max();
  }
  static __device__ __forceinline__ T apply(T a, T b) {
    if constexpr (std::is_floating_point<T>::value) {
      if (a != a) return a;
      if (b != b) return b;
      if (a == b) return signbit(a) ? a : b;
      return a < b ? a : b;
    } else {
      return a < b ? a : b;
    }
  }
};

// T <-> its bits zero-extended to 64 (the status value slot)
template <typename T> __device__ __forceinline__ unsigned long long to_bits64(T v) {
  if constexpr (sizeof(T) == 2) return (unsigned long long)__builtin_bit_cast(uint16_t, v);
  else if constexpr (sizeof(T) == 4) return (unsigned long long)__builtin_bit_cast(uint32_t, v);
  else return __builtin_bit_cast(unsigned long long, v);
}
template <typename T> __host__ __device__ __forceinline__ T from_bits64(unsigned long long b) {
  if constexpr (sizeof(T) == 2) return __builtin_bit_cast(T, uint16_t(b));
  else if constexpr (sizeof(T) == 4) return __builtin_bit_cast(T, uint32_t(b));
  else return __builtin_bit_cast(T, b);
}

__device__ __forceinline__ uint32_t ld_acquire_flag(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_flag(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct ScanArgs {
  const void *x;
  void *out;
  int64_t n;
  int64_t num_tiles;
  unsigned long long init_bits;
  int inclusive;
  int aligned16;      // x and out 16-byte aligned: whole tiles take vector loads
  int debug_skip;     // tile ids start at 1 (tile 0 never published: exercises the timeout)
  uint64_t timeout_ns;
  DevHeader *hdr;
  uint32_t *flags;                // [num_tiles]: 0, SCAN_FLAG_AGG, SCAN_FLAG_INC
  unsigned long long *agg_bits;   // [num_tiles]: the tile's aggregate, written before AGG
  unsigned long long *inc_bits;   // [num_tiles]: the inclusive prefix, written before INC
};

}  // namespace ak

namespace ak {

// Inclusive scan of one value per thread over the CTA under OP; `warp_tot`
// holds SCAN_BLOCK / 32 values.  Returns the thread's exclusive prefix (the
// identity for thread 0) and sets *total to the CTA's aggregate.
template <typename T, int OP>
__device__ __forceinline__ T cta_exclusive(T v, T *warp_tot, T *total) {
  using Op = ScanOp<T, OP>;
  constexpr int NW = SCAN_BLOCK / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = Op::apply(u, inc);
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NW ? warp_tot[lane] : Op::identity();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w = Op::apply(u, w);
    }
    if (lane < NW) warp_tot[lane] = w;  // inclusive over warps 0..lane
  }
  __syncthreads();
  *total = warp_tot[NW - 1];
  const T before_warp = warp == 0 ? Op::identity() : warp_tot[warp - 1];
  T ex = __shfl_up_sync(0xffffffffu, inc, 1);
  ex = lane == 0 ? before_warp : Op::apply(before_warp, ex);
  return ex;
}

// Bounded wait for a tile's flag; on expiry records AK_ERR_TIMEOUT and
// returns 0 (the caller then takes the identity and stops looking back).
__device__ __forceinline__ uint32_t scan_wait_flag(const uint32_t *p, uint64_t timeout_ns, DevHeader *hdr) {
  uint32_t f = ld_acquire_flag(p);
  if (f != 0) return f;
  const uint64_t t0 = globaltimer_ns();
  uint32_t spins = 0;
  while ((f = ld_acquire_flag(p)) == 0) {
    __nanosleep(64);
    if ((++spins & 15u) == 0 && globaltimer_ns() - t0 > timeout_ns) {
      set_error(hdr, AK_ERR_TIMEOUT);
      return 0;
    }
  }
  return f;
}

// Warp 0: the prefix of every tile before `tile` (identity for tile 0), found
// by looking back over windows of 32 predecessors.  In each window lane l
// holds tile j - l; the lanes up to the nearest inclusive prefix are combined
// with the earlier tile on the left, and the walk stops there.
template <typename T, int OP>
__device__ __forceinline__ T scan_look_back(const ScanArgs &a, int64_t tile) {
  using Op = ScanOp<T, OP>;
  const int lane = threadIdx.x & 31;
  T excl = Op::identity();
  for (int64_t j = tile - 1;; j -= 32) {
    const int64_t t = j - lane;
    bool stop = t < 0;  // nothing before tile 0
    T val = Op::identity();
    if (t >= 0) {
      const uint32_t f = scan_wait_flag(&a.flags[t], a.timeout_ns, a.hdr);
      if (f == SCAN_FLAG_INC) {
        val = from_bits64<T>(ld_relaxed(&a.inc_bits[t]));
        stop = true;
      } else if (f == SCAN_FLAG_AGG) {
        val = from_bits64<T>(ld_relaxed(&a.agg_bits[t]));
      } else {
        stop = true;  // timed out: identity
      }
    }
    const uint32_t stops = __ballot_sync(0xffffffffu, stop);
    const int last = stops ? __ffs(stops) - 1 : 31;  // nearest lane that ends the walk
    T w = lane <= last ? val : Op::identity();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_down_sync(0xffffffffu, w, o);
      if (lane + o < 32) w = Op::apply(u, w);  // lane + o holds the earlier tiles
    }
    excl = Op::apply(__shfl_sync(0xffffffffu, w, 0), excl);
    if (stops) return excl;
  }
}

template <typename T, int OP>
__global__ void __launch_bounds__(SCAN_BLOCK, 2) scan_kernel(ScanArgs a) {
  using Op = ScanOp<T, OP>;
  constexpr int PER_VEC = 16 / int(sizeof(T));
  constexpr int VECS = scan_vecs(int(sizeof(T)));
  constexpr int ITEMS = VECS * PER_VEC;
  constexpr int TILE = SCAN_BLOCK * ITEMS;
  __shared__ T s_warp[SCAN_BLOCK / 32];
  __shared__ T s_prefix;
  __shared__ int64_t s_tile;
  const int tid = threadIdx.x;
  // x and out may be the same array (in place): each thread reads its own run
  // before the CTA barriers and writes it after them; the next tile's run is
  // read before this tile's run is written, and the two never overlap
  const T *x = static_cast<const T *>(a.x);
  T *out = static_cast<T *>(a.out);
  const T init = from_bits64<T>(a.init_bits);
  // this thread's run of a tile into registers (identity past the end of the array)
  auto load_run = [&](int64_t tile, T (&v)[ITEMS]) {
    const int64_t base = tile * TILE;
    const int64_t tile_n = (a.n - base) < int64_t(TILE) ? (a.n - base) : int64_t(TILE);
    const int64_t first = base + int64_t(tid) * ITEMS;
    const int64_t end = base + tile_n;
    if (a.aligned16 && tile_n == TILE) {
      const uint4 *src = reinterpret_cast<const uint4 *>(x + first);
#pragma unroll
      for (int r = 0; r < VECS; ++r) {
        const uint4 q = src[r];
#pragma unroll
        for (int k = 0; k < PER_VEC; ++k) v[r * PER_VEC + k] = reinterpret_cast<const T *>(&q)[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) v[k] = first + k < end ? x[first + k] : Op::identity();
    }
  };
  if (tid == 0) s_tile = int64_t(atomicAdd(&a.hdr->tile_counter[0], 1u)) + (a.debug_skip ? 1 : 0);
  __syncthreads();
  int64_t tile = s_tile;
  T v[ITEMS];
  if (tile < a.num_tiles) load_run(tile, v);
  while (tile < a.num_tiles) {
    const int64_t base = tile * TILE;
    const int64_t tile_n = (a.n - base) < int64_t(TILE) ? (a.n - base) : int64_t(TILE);
    const int64_t first = base + int64_t(tid) * ITEMS;  // this thread's run of ITEMS
    const int64_t end = base + tile_n;
    const bool vec = a.aligned16 && tile_n == TILE;
    // 1. running prefix of the run, then the CTA scan of the run totals
#pragma unroll
    for (int k = 1; k < ITEMS; ++k) v[k] = Op::apply(v[k - 1], v[k]);
    T agg;
    const T run_ex = cta_exclusive<T, OP>(v[ITEMS - 1], s_warp, &agg);
    // 2. publish the aggregate and claim the next tile (its loads then fly
    //    while warp 0 looks back)
    if (tid == 0) {
      if (tile > 0) {
        st_relaxed(&a.agg_bits[tile], to_bits64(agg));
        st_release_flag(&a.flags[tile], SCAN_FLAG_AGG);
      }
      s_tile = int64_t(atomicAdd(&a.hdr->tile_counter[0], 1u)) + (a.debug_skip ? 1 : 0);
    }
    __syncthreads();
    const int64_t next = s_tile;
    // whole, aligned next tile: its run is loaded now as raw 16-byte vectors
    // (unpacked after this tile is written); otherwise it is loaded then
    uint4 nq[VECS];
    const bool next_vec = next < a.num_tiles && a.aligned16 && (a.n - next * TILE) >= int64_t(TILE);
    if (next_vec) {
      const uint4 *src = reinterpret_cast<const uint4 *>(x + next * TILE + int64_t(tid) * ITEMS);
#pragma unroll
      for (int r = 0; r < VECS; ++r) nq[r] = src[r];
    }
    // 3. look back, publish the inclusive prefix
    if (tid < 32) {
      T excl = Op::identity();
      if (tile > 0) excl = scan_look_back<T, OP>(a, tile);
      if (tid == 0) {
        st_relaxed(&a.inc_bits[tile], to_bits64(Op::apply(excl, agg)));
        st_release_flag(&a.flags[tile], SCAN_FLAG_INC);
        s_prefix = excl;
      }
    }
    __syncthreads();
    // 4. outputs: init (+) tile prefix (+) run prefix (+) the run so far
    const T lead = Op::apply(Op::apply(init, s_prefix), run_ex);
    T o[ITEMS];
    if (a.inclusive) {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) o[k] = Op::apply(lead, v[k]);
    } else {
      o[0] = lead;
#pragma unroll
      for (int k = 1; k < ITEMS; ++k) o[k] = Op::apply(lead, v[k - 1]);
    }
    if (vec) {
      uint4 *dst = reinterpret_cast<uint4 *>(out + first);
#pragma unroll
      for (int r = 0; r < VECS; ++r) {
        uint4 q;
#pragma unroll
        for (int k = 0; k < PER_VEC; ++k) reinterpret_cast<T *>(&q)[k] = o[r * PER_VEC + k];
        dst[r] = q;
      }
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k)
        if (first + k < end) out[first + k] = o[k];
    }
    if (next_vec) {
#pragma unroll
      for (int r = 0; r < VECS; ++r)
#pragma unroll
        for (int k = 0; k < PER_VEC; ++k) v[r * PER_VEC + k] = reinterpret_cast<const T *>(&nq[r])[k];
    } else if (next < a.num_tiles) {
      load_run(next, v);
    }
    tile = next;
    __syncthreads();  // s_tile, s_prefix and s_warp are rewritten by the next tile
  }
}

}  // namespace ak

namespace ak {
namespace {

inline size_t scan_align256(size_t x) { return (x + 255) & ~size_t(255); }

struct ScanLayout {
  int64_t tiles;
  size_t flags, agg, inc, total;  // byte offsets in the workspace (header at 0)
};

ScanLayout scan_layout(int64_t n, int key_bytes) {
  ScanLayout L;
  const int64_t tile = scan_tile(key_bytes);
  L.tiles = (n + tile - 1) / tile;
  size_t off = scan_align256(sizeof(DevHeader));
  L.flags = off;
  off += scan_align256(size_t(L.tiles) * 4);
  L.agg = off;
  off += scan_align256(size_t(L.tiles) * 8);
  L.inc = off;
  off += scan_align256(size_t(L.tiles) * 8);
  L.total = off;
  return L;
}

int scan_key_bytes(int kd) {
  switch (kd) {
    case AK_U16: case AK_I16: return 2;
    case AK_U32: case AK_I32: case AK_F32: return 4;
    case AK_U64: case AK_I64: case AK_F64: return 8;
  }
  return 0;
}

// Bits of the operator's identity for a key type (the default start value).
unsigned long long scan_identity_bits(int kd, int op) {
  const bool fl = kd == AK_F32 || kd == AK_F64;
  const int bits = 8 * scan_key_bytes(kd);
  const unsigned long long ones = bits == 64 ? ~0ull : ((1ull << bits) - 1);
  const unsigned long long top = 1ull << (bits - 1);  // sign bit
  const bool sgn = kd == AK_I16 || kd == AK_I32 || kd == AK_I64;
  const unsigned long long inf = kd == AK_F32 ? 0x7F800000ull : 0x7FF0000000000000ull;
  switch (op) {
    case AK_SCAN_ADD: return fl ? top : 0ull;                           // -0.0 or 0
    case AK_SCAN_MAX: return fl ? (inf | top) : (sgn ? top : 0ull);     // -Inf or the lowest
    default: return fl ? inf : (sgn ? (ones >> 1) : ones);              // +Inf or the highest
  }
}

// Resident CTAs of one scan kernel on a device (cached per kernel and device).
int scan_resident(const void *fn, int dev) {
  static std::mutex mu;
  static const void *fns[64];
  static int devs[64], vals[64], used = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (fns[i] == fn && devs[i] == dev) return vals[i];
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SCAN_BLOCK, 0) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int total = per_sm * sms;
  if (used < 64 && total > 0) {
    fns[used] = fn;
    devs[used] = dev;
    vals[used++] = total;
  }
  return total;
}

template <typename T, int OP>
ak_status scan_launch(ScanArgs &a, cudaStream_t st) {
  auto *fn = scan_kernel<T, OP>;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AK_ERR_CUDA;
  const int resident = scan_resident(reinterpret_cast<const void *>(fn), dev);
  if (resident <= 0) return AK_ERR_CUDA;
  const int grid = int(a.num_tiles < resident ? a.num_tiles : resident);
  fn<<<grid, SCAN_BLOCK, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? AK_OK : AK_ERR_CUDA;
}

template <typename T>
ak_status scan_op_dispatch(int op, ScanArgs &a, cudaStream_t st) {
  switch (op) {
    case AK_SCAN_ADD: return scan_launch<T, AK_SCAN_ADD>(a, st);
    case AK_SCAN_MAX: return scan_launch<T, AK_SCAN_MAX>(a, st);
    case AK_SCAN_MIN: return scan_launch<T, AK_SCAN_MIN>(a, st);
  }
  return AK_ERR_INVALID_ARG;
}

ak_status scan_dispatch(int kd, int op, ScanArgs &a, cudaStream_t st) {
  switch (kd) {
    case AK_U16: return scan_op_dispatch<uint16_t>(op, a, st);
    case AK_I16: return scan_op_dispatch<int16_t>(op, a, st);
    case AK_U32: return scan_op_dispatch<uint32_t>(op, a, st);
    case AK_I32: return scan_op_dispatch<int32_t>(op, a, st);
    case AK_U64: return scan_op_dispatch<uint64_t>(op, a, st);
    case AK_I64: return scan_op_dispatch<int64_t>(op, a, st);
    case AK_F32: return scan_op_dispatch<float>(op, a, st);
    case AK_F64: return scan_op_dispatch<double>(op, a, st);
  }
  return AK_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace ak

extern "C" {

ak_status ak_accumulate_temp_bytes(int64_t n, ak_dtype kd, size_t *bytes) {
  if (kd == AK_F16 || kd == AK_BF16) return AK_ERR_UNSUPPORTED;  // 16-bit float sums: no rounding defined
  const int kb = ak::scan_key_bytes(int(kd));
  if (!bytes || n < 0 || kb == 0) return AK_ERR_INVALID_ARG;
  *bytes = ak::scan_layout(n, kb).total;
  return AK_OK;
}

ak_status ak_accumulate(const void *d_x, void *d_out, int64_t n, ak_dtype kd, ak_scan_op op, int inclusive,
                        const void *h_init, void *d_temp, size_t temp_bytes, ak_stream_t stream,
                        const ak_options *opt) {
  if (kd == AK_F16 || kd == AK_BF16) return AK_ERR_UNSUPPORTED;  // 16-bit float sums: no rounding defined
  const int kb = ak::scan_key_bytes(int(kd));
  ak_options o;
  if (n < 0 || kb == 0 || op < AK_SCAN_ADD || op > AK_SCAN_MIN || (inclusive != 0 && inclusive != 1) ||
      !ak::resolve_options(opt, &o))
    return AK_ERR_INVALID_ARG;
  if (n == 0) return AK_OK;
  auto misaligned = [](const void *p, uintptr_t al) { return (reinterpret_cast<uintptr_t>(p) % al) != 0; };
  if (!d_x || !d_out || misaligned(d_x, kb) || misaligned(d_out, kb)) return AK_ERR_INVALID_ARG;
  if (d_temp && misaligned(d_temp, 256)) return AK_ERR_INVALID_ARG;
  const ak::ScanLayout L = ak::scan_layout(n, kb);
  if (!d_temp || temp_bytes < L.total) return AK_ERR_WORKSPACE_TOO_SMALL;
  ak::ScanArgs a{};
  a.x = d_x;
  a.out = d_out;
  a.n = n;
  a.num_tiles = L.tiles;
  a.init_bits = 0;
  if (h_init) std::memcpy(&a.init_bits, h_init, size_t(kb));  // little-endian: low bytes hold the value
  else a.init_bits = ak::scan_identity_bits(int(kd), int(op));
  a.inclusive = inclusive;
  a.aligned16 = !misaligned(d_x, 16) && !misaligned(d_out, 16);
  a.debug_skip = (o.debug_flags & AK_DEBUG_SKIP_FIRST_TILE) ? 1 : 0;
  a.timeout_ns = o.timeout_ns;
  char *t = static_cast<char *>(d_temp);
  a.hdr = reinterpret_cast<ak::DevHeader *>(t);
  a.flags = reinterpret_cast<uint32_t *>(t + L.flags);
  a.agg_bits = reinterpret_cast<unsigned long long *>(t + L.agg);
  a.inc_bits = reinterpret_cast<unsigned long long *>(t + L.inc);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // header (status, tile counter) and the flags start at zero; values need no clearing
  if (cudaMemsetAsync(t, 0, L.agg, st) != cudaSuccess) return AK_ERR_CUDA;
  return ak::scan_dispatch(int(kd), int(op), a, st);
}

}  // extern "C"
