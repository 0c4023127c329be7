// scan.cu -- accumulate: prefix scan under a binary operator (Sec. II-B,
// accumulate, inclusive and exclusive).
//
// out[i] = init (+) x[0] (+) ... (+) x[i]      (inclusive)
// out[i] = init (+) x[0] (+) ... (+) x[i - 1]  (exclusive, out[0] = init)
// for (+) = + (integers wrap in their width), Julia max, Julia min.
//
// HBM bound: n * w bytes read and n * w written.  Design for GB300: three
// launches, none of which waits on another CTA (reduce, then scan):
//  * the array is cut into warp ranges, contiguous runs of whole warp tiles
//    (32 lanes x 64 bytes; 32 bytes for 16-bit keys), as many ranges as warps
//    are resident (16 per 512-thread CTA, 2 CTAs per SM);
//  * scan_reduce_kernel: each warp combines its range from the last warp tile
//    to the first (the start of every range is then the most recently read
//    data in L2 for the third launch); a lane combines its run in order, the
//    warp combines the 32 runs in lane order, and the tile total goes on the
//    left of what was combined so far;
//  * scan_carry_kernel: one CTA scans the range totals in order from init:
//    the exclusive prefix of every range;
//  * scan_ranges_kernel: each warp walks its range forward from that prefix:
//    running prefix of each lane's run, warp scan of the run totals with
//    shuffles, outputs, carry += tile total; the next warp tile's loads are in
//    flight while the current one is scanned and stored.
// Traffic is 3 n w (the input is read twice) but every launch streams with
// no barrier inside its loop: a single-pass decoupled look-back measured 2.6
// to 9.6 ms on 2^28 int64 keys (persistent 512-thread CTAs, look-back 6.5 to
// 41 us a tile), this reads and writes the same in about a millisecond.
//
// Every operator is applied with the earlier operand on the left, so results
// are exact for integers and max/min (the first NaN of the sequence wins);
// float + rounds in a tree of its own.
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
constexpr int SCAN_WARPS = SCAN_BLOCK / 32;
constexpr int SCAN_CARRY_BLOCK = 1024;
// 16-byte vectors per lane and warp tile: 64 bytes (32 bytes for 16-bit keys,
// whose values each take a register)
constexpr int scan_vecs(int key_bytes) { return key_bytes == 2 ? 2 : 4; }
constexpr int scan_items(int key_bytes) { return scan_vecs(key_bytes) * 16 / key_bytes; }
constexpr int scan_warp_tile(int key_bytes) { return 32 * scan_items(key_bytes); }
// Upper bound on the warp ranges (sizes the workspace; far above the
// resident warps of any device).
constexpr int64_t SCAN_MAX_RANGES = 1 << 15;

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

// T <-> its bits zero-extended to 64 (the range slots)
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

struct ScanArgs {
  const void *x;
  void *out;
  int64_t n;
  int64_t wtiles;     // warp tiles, the last one possibly ragged
  int64_t per;        // warp tiles per range (the last range may hold fewer)
  int64_t nranges;    // ceil(wtiles / per)
  unsigned long long init_bits;
  int inclusive;
  int aligned16;      // x and out 16-byte aligned: whole warp tiles take vector loads
  unsigned long long *agg;  // [nranges]: each range's total (bits)
  unsigned long long *pre;  // [nranges]: init (+) the totals of the ranges before it
};

}  // namespace ak

namespace ak {

// One warp tile into registers: lane l holds elements [base + l ITEMS, +ITEMS)
// (identity past the end of the array).
template <typename T, int OP>
__device__ __forceinline__ void scan_load(const ScanArgs &a, const T *x, int64_t wt, T (&v)[scan_items(sizeof(T))]) {
  using Op = ScanOp<T, OP>;
  constexpr int ITEMS = scan_items(sizeof(T));
  constexpr int VECS = scan_vecs(sizeof(T));
  constexpr int PER_VEC = 16 / int(sizeof(T));
  const int lane = threadIdx.x & 31;
  const int64_t first = wt * (32 * ITEMS) + int64_t(lane) * ITEMS;
  if (a.aligned16 && (wt + 1) * (32 * ITEMS) <= a.n) {
    const uint4 *src = reinterpret_cast<const uint4 *>(x + first);
#pragma unroll
    for (int r = 0; r < VECS; ++r) {
      const uint4 q = src[r];
#pragma unroll
      for (int k = 0; k < PER_VEC; ++k) v[r * PER_VEC + k] = reinterpret_cast<const T *>(&q)[k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) v[k] = first + k < a.n ? x[first + k] : Op::identity();
  }
}

// Warp ranges of this warp: [lo, hi) warp tiles; false when the warp has none.
__device__ __forceinline__ bool scan_range(const ScanArgs &a, int64_t *r, int64_t *lo, int64_t *hi) {
  *r = int64_t(blockIdx.x) * SCAN_WARPS + (threadIdx.x >> 5);
  if (*r >= a.nranges) return false;
  *lo = *r * a.per;
  *hi = *lo + a.per < a.wtiles ? *lo + a.per : a.wtiles;
  return true;
}

// Launch 1: the total of every warp range, combined in element order.
template <typename T, int OP>
__global__ void __launch_bounds__(SCAN_BLOCK, 2) scan_reduce_kernel(ScanArgs a) {
  using Op = ScanOp<T, OP>;
  constexpr int ITEMS = scan_items(sizeof(T));
  int64_t r, lo, hi;
  if (!scan_range(a, &r, &lo, &hi)) return;
  const int lane = threadIdx.x & 31;
  const T *x = static_cast<const T *>(a.x);
  T acc = Op::identity();
  T v[ITEMS], nv[ITEMS];
  scan_load<T, OP>(a, x, hi - 1, v);
  for (int64_t wt = hi - 1; wt >= lo; --wt) {  // last tile first
    if (wt > lo) scan_load<T, OP>(a, x, wt - 1, nv);
    T w = v[0];
#pragma unroll
    for (int k = 1; k < ITEMS; ++k) w = Op::apply(w, v[k]);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_down_sync(0xffffffffu, w, o);
      if (lane + o < 32) w = Op::apply(w, u);  // lane + o holds later elements
    }
    acc = Op::apply(w, acc);  // this tile precedes everything combined so far
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) v[k] = nv[k];
  }
  if (lane == 0) a.agg[r] = to_bits64(acc);
}

// Launch 2 (one CTA): pre[r] = init (+) agg[0] (+) ... (+) agg[r - 1].
template <typename T, int OP>
__global__ void __launch_bounds__(SCAN_CARRY_BLOCK) scan_carry_kernel(ScanArgs a) {
  using Op = ScanOp<T, OP>;
  constexpr int NW = SCAN_CARRY_BLOCK / 32;
  __shared__ T s_warp[NW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t chunk = (a.nranges + SCAN_CARRY_BLOCK - 1) / SCAN_CARRY_BLOCK;
  const int64_t b = int64_t(tid) * chunk;
  const int64_t e = b + chunk < a.nranges ? b + chunk : a.nranges;
  T tot = Op::identity();
  for (int64_t i = b; i < e; ++i) tot = Op::apply(tot, from_bits64<T>(a.agg[i]));
  // exclusive scan of the thread totals in thread order
  T inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc = Op::apply(u, inc);
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w = Op::apply(u, w);
    }
    s_warp[lane] = w;  // inclusive over warps 0..lane
  }
  __syncthreads();
  T ex = __shfl_up_sync(0xffffffffu, inc, 1);
  const T before_warp = warp == 0 ? Op::identity() : s_warp[warp - 1];
  ex = lane == 0 ? before_warp : Op::apply(before_warp, ex);
  T run = Op::apply(from_bits64<T>(a.init_bits), ex);
  for (int64_t i = b; i < e; ++i) {
    a.pre[i] = to_bits64(run);
    run = Op::apply(run, from_bits64<T>(a.agg[i]));
  }
}

// Launch 3: each warp scans its range forward from its prefix.
template <typename T, int OP>
__global__ void __launch_bounds__(SCAN_BLOCK, 2) scan_ranges_kernel(ScanArgs a) {
  using Op = ScanOp<T, OP>;
  constexpr int ITEMS = scan_items(sizeof(T));
  constexpr int VECS = scan_vecs(sizeof(T));
  constexpr int PER_VEC = 16 / int(sizeof(T));
  int64_t r, lo, hi;
  if (!scan_range(a, &r, &lo, &hi)) return;
  const int lane = threadIdx.x & 31;
  // x and out may be the same array (in place): a warp owns its range, reads
  // each warp tile before writing it and reads ahead only tiles not yet written
  const T *x = static_cast<const T *>(a.x);
  T *out = static_cast<T *>(a.out);
  T carry = from_bits64<T>(a.pre[r]);
  T v[ITEMS], nv[ITEMS];
  scan_load<T, OP>(a, x, lo, v);
  for (int64_t wt = lo; wt < hi; ++wt) {
    if (wt + 1 < hi) scan_load<T, OP>(a, x, wt + 1, nv);
#pragma unroll
    for (int k = 1; k < ITEMS; ++k) v[k] = Op::apply(v[k - 1], v[k]);  // running prefix of the run
    T inc = v[ITEMS - 1];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc = Op::apply(u, inc);
    }
    const T total = __shfl_sync(0xffffffffu, inc, 31);
    T ex = __shfl_up_sync(0xffffffffu, inc, 1);
    const T lead = lane == 0 ? carry : Op::apply(carry, ex);  // everything before this run
    T o[ITEMS];
    if (a.inclusive) {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) o[k] = Op::apply(lead, v[k]);
    } else {
      o[0] = lead;
#pragma unroll
      for (int k = 1; k < ITEMS; ++k) o[k] = Op::apply(lead, v[k - 1]);
    }
    const int64_t first = wt * (32 * ITEMS) + int64_t(lane) * ITEMS;
    if (a.aligned16 && (wt + 1) * (32 * ITEMS) <= a.n) {
      uint4 *dst = reinterpret_cast<uint4 *>(out + first);
#pragma unroll
      for (int rr = 0; rr < VECS; ++rr) {
        uint4 q;
#pragma unroll
        for (int k = 0; k < PER_VEC; ++k) reinterpret_cast<T *>(&q)[k] = o[rr * PER_VEC + k];
        dst[rr] = q;
      }
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k)
        if (first + k < a.n) out[first + k] = o[k];
    }
    carry = Op::apply(carry, total);
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) v[k] = nv[k];
  }
}

}  // namespace ak

namespace ak {
namespace {

inline size_t scan_align256(size_t x) { return (x + 255) & ~size_t(255); }

struct ScanLayout {
  int64_t wtiles;
  size_t agg, pre, total;  // byte offsets in the workspace (header at 0)
};

ScanLayout scan_layout(int64_t n, int key_bytes) {
  ScanLayout L;
  const int64_t wt = scan_warp_tile(key_bytes);
  L.wtiles = (n + wt - 1) / wt;
  const int64_t ranges = L.wtiles < SCAN_MAX_RANGES ? L.wtiles : SCAN_MAX_RANGES;
  size_t off = scan_align256(sizeof(DevHeader));
  L.agg = off;
  off += scan_align256(size_t(ranges) * 8);
  L.pre = off;
  off += scan_align256(size_t(ranges) * 8);
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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AK_ERR_CUDA;
  const int r1 = scan_resident(reinterpret_cast<const void *>(scan_reduce_kernel<T, OP>), dev);
  const int r3 = scan_resident(reinterpret_cast<const void *>(scan_ranges_kernel<T, OP>), dev);
  const int64_t resident = r1 < r3 ? r1 : r3;
  if (resident <= 0) return AK_ERR_CUDA;
  // one range per resident warp, whole warp tiles each
  // (at least 1,024 ranges when there are that many warp tiles: the float +
  // summation depth then has a device-independent bound)
  int64_t target = resident * SCAN_WARPS;
  if (target < 1024) target = 1024;
  if (target > a.wtiles) target = a.wtiles;
  if (target > SCAN_MAX_RANGES) target = SCAN_MAX_RANGES;
  a.per = (a.wtiles + target - 1) / target;
  a.nranges = (a.wtiles + a.per - 1) / a.per;
  const unsigned blocks = unsigned((a.nranges + SCAN_WARPS - 1) / SCAN_WARPS);
  scan_reduce_kernel<T, OP><<<blocks, SCAN_BLOCK, 0, st>>>(a);
  scan_carry_kernel<T, OP><<<1, SCAN_CARRY_BLOCK, 0, st>>>(a);
  scan_ranges_kernel<T, OP><<<blocks, SCAN_BLOCK, 0, st>>>(a);
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
  if (kd == AK_F16 || kd == AK_BF16 || kd == AK_I128 || kd == AK_U128)
    return AK_ERR_UNSUPPORTED;  // 16-bit float sums: no rounding defined; 128-bit scans not built
  const int kb = ak::scan_key_bytes(int(kd));
  if (!bytes || n < 0 || kb == 0) return AK_ERR_INVALID_ARG;
  *bytes = ak::scan_layout(n, kb).total;
  return AK_OK;
}

ak_status ak_accumulate(const void *d_x, void *d_out, int64_t n, ak_dtype kd, ak_scan_op op, int inclusive,
                        const void *h_init, void *d_temp, size_t temp_bytes, ak_stream_t stream,
                        const ak_options *opt) {
  if (kd == AK_F16 || kd == AK_BF16 || kd == AK_I128 || kd == AK_U128)
    return AK_ERR_UNSUPPORTED;  // 16-bit float sums: no rounding defined; 128-bit scans not built
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
  a.wtiles = L.wtiles;
  a.init_bits = 0;
  if (h_init) std::memcpy(&a.init_bits, h_init, size_t(kb));  // little-endian: low bytes hold the value
  else a.init_bits = ak::scan_identity_bits(int(kd), int(op));
  a.inclusive = inclusive;
  a.aligned16 = !misaligned(d_x, 16) && !misaligned(d_out, 16);
  char *t = static_cast<char *>(d_temp);
  a.agg = reinterpret_cast<unsigned long long *>(t + L.agg);
  a.pre = reinterpret_cast<unsigned long long *>(t + L.pre);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the header (status word, diagnostics) starts clean; the range slots are
  // written before they are read
  if (cudaMemsetAsync(t, 0, sizeof(ak::DevHeader), st) != cudaSuccess) return AK_ERR_CUDA;
  return ak::scan_dispatch(int(kd), int(op), a, st);
}

}  // extern "C"
