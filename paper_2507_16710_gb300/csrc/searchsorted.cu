// searchsorted.cu -- batched binary search over a sorted key array (Sec. II-B,
// searchsortedfirst / searchsortedlast), in the sort's order (Julia isless or
// its reverse).
//
// Every comparison is made on the radix key of common.cuh: r(a) < r(b) exactly
// when a comes before b in the order (all NaNs tie, -0.0 before +0.0), so the
// search is plain unsigned bisection.  One thread answers one query at a time.
// A query's answer is the length of the prefix of v on which a predicate holds
// ("comes before x" for the first index, "x does not come before it" for the
// last one); on a sorted v that prefix is where bisection lands.
//
// Queries go in tiles of 4,096 per CTA iteration, staged as radix keys in
// shared memory; a tile whose keys are in the order of v (checked on the
// spot: no flag from the caller, no workspace) is answered by a merge-like
// scheme, any other tile by bisection per query.
//
// Bisection (unsorted tiles), two levels, latency-bound on GB300:
//  * a table of K pivot keys in shared memory (16 KB: K = 8192, 4096, 2048, 1024 for
//    2-, 4-, 8-, 16-byte keys), v at positions P_i = floor(i n / (K + 1)),
//    i = 1..K, loaded once per CTA; the table narrows each query to the stretch
//    (P_c, P_{c+1}] of about n / (K + 1) keys with no global access;
//  * bisection in global memory over that stretch, log2(n / K) dependent loads,
//    the upper ones shared by many queries and held in the 129 MB L2.
// Sorted tiles: the answers of the tile lie between those of its first and
// last query.  Those two come from the table and then a 256-way search by
// half of the CTA each (a round of 256 independent loads narrows a stretch
// 257-fold: two rounds for 2^27 keys; SS_HALF-way in general); the keys of v between them are read
// once, coalesced, into a 64 KB shared window, chunk after chunk, and each
// query bisects the chunk that holds its answer.  v is then read about once
// over all the tiles: HBM bound instead of latency bound.  A stretch above
// eight windows (queries sparse in v) is bisected in global memory instead.
// Persistent CTAs (a grid of the resident count) walk the tiles, so each CTA
// loads its table once.  Reads of x and writes of out are coalesced.
//
// Bounds: K <= n - 1, so the pivots strictly increase and (P_c, P_{c+1}] stays
// inside [0, n) whatever v holds; an unsorted v gives unspecified answers in
// [0, n] (first) or [-1, n - 1] (last) and no access outside v[0, n): every
// search keeps 0 <= lo <= hi <= n and reads only v[lo, hi).
#include <mutex>

#include "common.cuh"

namespace ak {

constexpr int SS_BLOCK = 512;
constexpr int SS_MIN_BLOCKS = 2;            // CTAs per SM the registers are sized for
constexpr int SS_TABLE_BYTES = 16384;
constexpr int SS_TILE = 4096;               // queries per CTA iteration
constexpr int SS_WINDOW_BYTES = 65536;      // shared window of v for a sorted tile
constexpr int SS_HALF = SS_BLOCK / 2;       // probes per round of a tile-bound search
constexpr int SS_PARTS = SS_HALF + 1;       // a round narrows a stretch SS_PARTS-fold
constexpr int SS_WINDOW_CHUNKS = 8;         // windows a sorted tile reads before it bisects in global memory

template <typename U>
constexpr size_t ss_smem_bytes() {
  return size_t(SS_TABLE_BYTES) + size_t(SS_TILE) * sizeof(U) + size_t(SS_WINDOW_BYTES);
}

// floor(i * n / parts) as i * q + floor(i * r / parts), n = q * parts + r:
// exact, and no intermediate exceeds n or parts^2.
__device__ __forceinline__ int64_t ss_pivot(int64_t i, int64_t q, int64_t r, int64_t parts) {
  return i * q + (i * r) / parts;
}

template <bool LAST, typename U>
__device__ __forceinline__ bool ss_in_prefix(U e, U key) {  // holds on a prefix of a sorted v
  return LAST ? e <= key : e < key;
}

// The stretch [lo, hi) of v the table leaves for `key`: everything before lo
// is in the prefix, nothing from hi on.
template <bool LAST, typename U>
__device__ __forceinline__ void ss_table(const U *s_t, int K, int64_t n, int64_t q, int64_t r, int64_t parts, U key,
                                         int64_t *lo, int64_t *hi) {
  int c = 0, len = K;  // c = table entries in the prefix
  while (len > 0) {
    const int half = len >> 1;
    if (ss_in_prefix<LAST>(s_t[c + half], key)) {
      c += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  // pivot c (table entry c - 1) is in the prefix, pivot c + 1 is not
  *lo = c == 0 ? 0 : ss_pivot(c, q, r, parts) + 1;
  *hi = c == K ? n : ss_pivot(c + 1, q, r, parts);
}

// Prefix length of `key` in v by bisection of [lo, hi) in global memory.
template <int KIND, bool LAST, typename U>
__device__ __forceinline__ int64_t ss_bisect_global(const U *__restrict__ v, U flip, U key, int64_t lo, int64_t hi) {
  int64_t span = hi - lo;
  while (span > 0) {
    const int64_t half = span >> 1;
    if (ss_in_prefix<LAST>(radix_key_t<KIND>(v[lo + half], flip), key)) {
      lo += half + 1;
      span -= half + 1;
    } else {
      span = half;
    }
  }
  return lo;
}

template <typename U, int KIND, bool LAST>
__global__ void __launch_bounds__(SS_BLOCK, SS_MIN_BLOCKS) searchsorted_kernel(const U *__restrict__ v, int64_t n,
                                                                   const U *__restrict__ x, int64_t m, U flip, int K,
                                                                   int64_t *__restrict__ out) {
  constexpr int WINDOW = SS_WINDOW_BYTES / int(sizeof(U));
  extern __shared__ __align__(16) uint8_t ss_smem[];
  U *s_t = reinterpret_cast<U *>(ss_smem);                                  // [TABLE] pivots
  U *s_x = reinterpret_cast<U *>(ss_smem + SS_TABLE_BYTES);                 // [SS_TILE] query radix keys
  U *s_w = reinterpret_cast<U *>(ss_smem + SS_TABLE_BYTES + SS_TILE * sizeof(U));  // [WINDOW] of v
  __shared__ long long s_lo[2], s_hi[2];  // search state of the first / last query of a tile
  __shared__ int s_cnt[2];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t parts = int64_t(K) + 1, q = n / parts, r = n % parts;
  for (int i = tid; i < K; i += SS_BLOCK) s_t[i] = radix_key_t<KIND>(v[ss_pivot(i + 1, q, r, parts)], flip);
  const int64_t ntiles = (m + SS_TILE - 1) / SS_TILE;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t base = t * SS_TILE;
    const int cnt = int((m - base) < SS_TILE ? (m - base) : SS_TILE);
    __syncthreads();  // the table is loaded; the previous tile's buffers are free
    for (int i = tid; i < cnt; i += SS_BLOCK) s_x[i] = radix_key_t<KIND>(x[base + i], flip);
    __syncthreads();
    bool down = false;  // a descent inside the tile: it is not in v's order
    for (int i = tid + 1; i < cnt; i += SS_BLOCK) down |= s_x[i] < s_x[i - 1];
    const bool sorted = __syncthreads_or(down) == 0;
    if (!sorted) {  // bisection per query
      for (int i = tid; i < cnt; i += SS_BLOCK) {
        const U key = s_x[i];
        int64_t lo, hi;
        ss_table<LAST>(s_t, K, n, q, r, parts, key, &lo, &hi);
        const int64_t a = ss_bisect_global<KIND, LAST>(v, flip, key, lo, hi);
        out[base + i] = LAST ? a - 1 : a;
      }
      continue;
    }
    // answers of the first and last query: table, then SS_HALF-way rounds (the
    // first half of the threads for the first query, the second for the last)
    const int g = tid / SS_HALF, j = tid % SS_HALF;
    const U gkey = s_x[g ? cnt - 1 : 0];
    if (j == 0) {
      int64_t lo, hi;
      ss_table<LAST>(s_t, K, n, q, r, parts, gkey, &lo, &hi);
      s_lo[g] = lo;
      s_hi[g] = hi;
      s_cnt[g] = 0;
    }
    __syncthreads();
    for (;;) {
      const int64_t a = s_lo[g], len = s_hi[g] - a;
      const bool live = len > 0;
      bool p = false;
      if (live) {
        // len <= SS_HALF: probe every key; else SS_HALF probes at
        // a + floor((j+1) len / SS_PARTS), strictly increasing, all below a + len
        const int64_t pos = len <= SS_HALF ? a + j : a + ((j + 1) * len) / SS_PARTS;
        if (len > SS_HALF || j < len) p = ss_in_prefix<LAST>(radix_key_t<KIND>(v[pos], flip), gkey);
      }
      const uint32_t b = __ballot_sync(0xffffffffu, p);
      if (lane == 0 && b) atomicAdd(&s_cnt[g], __popc(b));
      const bool any_live = __syncthreads_or(live);
      if (!any_live) break;
      if (j == 0 && live) {  // probes 0..c-1 are in the prefix, probe c is not
        const int c = s_cnt[g];
        if (len <= SS_HALF) {
          s_lo[g] = a + c;
          s_hi[g] = a + c;
        } else {
          const int64_t nlo = c == 0 ? a : a + (int64_t(c) * len) / SS_PARTS + 1;
          const int64_t nhi = c == SS_HALF ? a + len : a + (int64_t(c + 1) * len) / SS_PARTS;
          s_lo[g] = nlo;
          s_hi[g] = nhi;
        }
      }
      if (j == 0) s_cnt[g] = 0;
      __syncthreads();
    }
    const int64_t wlo = s_lo[0], whi = s_lo[1];  // every answer of the tile lies in [wlo, whi]
    const int64_t wn = whi - wlo;
    if (wn <= int64_t(SS_WINDOW_CHUNKS) * WINDOW) {
      // the keys between the bounds in chunks of the window, in order: a
      // query's answer lies in the first chunk whose last key is outside its
      // prefix (past every chunk: whi).  (Runs of consecutive queries per
      // thread, galloping from the previous answer, measured 12% slower:
      // bank conflicts on the staged queries and divergent gallops.)
      int64_t ans[SS_TILE / SS_BLOCK];
#pragma unroll
      for (int k = 0; k < SS_TILE / SS_BLOCK; ++k) ans[k] = -1;
      for (int64_t c0 = 0; c0 < wn; c0 += WINDOW) {
        const int cl = int((wn - c0) < WINDOW ? (wn - c0) : WINDOW);
        if (c0 > 0) __syncthreads();  // the previous chunk is no longer read
        for (int i = tid; i < cl; i += SS_BLOCK) s_w[i] = radix_key_t<KIND>(v[wlo + c0 + i], flip);
        __syncthreads();
        const U last_key = s_w[cl - 1];
#pragma unroll
        for (int k = 0; k < SS_TILE / SS_BLOCK; ++k) {
          const int i = tid + k * SS_BLOCK;
          if (i < cnt && ans[k] < 0) {
            const U key = s_x[i];
            if (!ss_in_prefix<LAST>(last_key, key)) {
              int lo = 0, span = cl - 1;  // the chunk's last key is known to be outside
              while (span > 0) {
                const int half = span >> 1;
                if (ss_in_prefix<LAST>(s_w[lo + half], key)) {
                  lo += half + 1;
                  span -= half + 1;
                } else {
                  span = half;
                }
              }
              ans[k] = wlo + c0 + lo;
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < SS_TILE / SS_BLOCK; ++k) {
        const int i = tid + k * SS_BLOCK;
        if (i < cnt) {
          const int64_t a = ans[k] < 0 ? (wn > 0 ? whi : wlo) : ans[k];
          out[base + i] = LAST ? a - 1 : a;
        }
      }
    } else {  // queries sparse in v: bisection in global memory between the tile's bounds
      for (int i = tid; i < cnt; i += SS_BLOCK) {
        const int64_t a = ss_bisect_global<KIND, LAST>(v, flip, s_x[i], wlo, whi);
        out[base + i] = LAST ? a - 1 : a;
      }
    }
  }
}

namespace {

// Resident CTAs per SM of one kernel on the current device (cached: the
// occupancy query is a host computation but not free).
int ss_resident_ctas(const void *fn, int dev, size_t smem) {
  static std::mutex mu;
  static const void *fns[64];
  static int devs[64], vals[64], used = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (fns[i] == fn && devs[i] == dev) return vals[i];
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SS_BLOCK, smem) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const int total = per_sm * sms;
  if (used < 64 && total > 0) {
    fns[used] = fn;
    devs[used] = dev;
    vals[used++] = total;
  }
  return total;
}

template <typename U, int KIND, bool LAST>
ak_status ss_launch(const void *v, int64_t n, const void *x, int64_t m, bool desc, int64_t *out,
                    cudaStream_t stream) {
  constexpr int TABLE = SS_TABLE_BYTES / int(sizeof(U));
  constexpr size_t SMEM = ss_smem_bytes<U>();
  auto *fn = searchsorted_kernel<U, KIND, LAST>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(SMEM)) != cudaSuccess)
    return AK_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AK_ERR_CUDA;
  const int resident = ss_resident_ctas(reinterpret_cast<const void *>(fn), dev, SMEM);
  if (resident <= 0) return AK_ERR_CUDA;
  const int64_t want = (m + SS_TILE - 1) / SS_TILE;
  const int grid = int(want < resident ? want : resident);
  const int K = int(n - 1 < TABLE ? (n > 0 ? n - 1 : 0) : TABLE);
  const U flip = desc ? U(~U(0)) : U(0);
  fn<<<grid, SS_BLOCK, SMEM, stream>>>(static_cast<const U *>(v), n, static_cast<const U *>(x), m, flip, K, out);
  return cudaGetLastError() == cudaSuccess ? AK_OK : AK_ERR_CUDA;
}

template <bool LAST>
ak_status ss_dispatch(const void *v, int64_t n, const void *x, int64_t m, int kd, bool desc, int64_t *out,
                      cudaStream_t st) {
  switch (kd) {
    case AK_U16: return ss_launch<uint16_t, KIND_UINT, LAST>(v, n, x, m, desc, out, st);
    case AK_I16: return ss_launch<uint16_t, KIND_SINT, LAST>(v, n, x, m, desc, out, st);
    case AK_U32: return ss_launch<uint32_t, KIND_UINT, LAST>(v, n, x, m, desc, out, st);
    case AK_I32: return ss_launch<uint32_t, KIND_SINT, LAST>(v, n, x, m, desc, out, st);
    case AK_F32: return ss_launch<uint32_t, KIND_FLOAT, LAST>(v, n, x, m, desc, out, st);
    case AK_U64: return ss_launch<uint64_t, KIND_UINT, LAST>(v, n, x, m, desc, out, st);
    case AK_I64: return ss_launch<uint64_t, KIND_SINT, LAST>(v, n, x, m, desc, out, st);
    case AK_F64: return ss_launch<uint64_t, KIND_FLOAT, LAST>(v, n, x, m, desc, out, st);
    case AK_F16: return ss_launch<uint16_t, KIND_FLOAT, LAST>(v, n, x, m, desc, out, st);
    case AK_BF16: return ss_launch<uint16_t, KIND_BF16, LAST>(v, n, x, m, desc, out, st);
    case AK_U128: return ss_launch<u128, KIND_UINT, LAST>(v, n, x, m, desc, out, st);
    case AK_I128: return ss_launch<u128, KIND_SINT, LAST>(v, n, x, m, desc, out, st);
  }
  return AK_ERR_INVALID_ARG;
}

int ss_key_bytes(int kd) {
  switch (kd) {
    case AK_U16: case AK_I16: case AK_F16: case AK_BF16: return 2;
    case AK_U32: case AK_I32: case AK_F32: return 4;
    case AK_U64: case AK_I64: case AK_F64: return 8;
    case AK_U128: case AK_I128: return 16;
  }
  return 0;
}

template <bool LAST>
ak_status ss_entry(const void *d_v, int64_t n, const void *d_x, int64_t m, ak_dtype kd, ak_order order,
                   int64_t *d_out, ak_stream_t stream) {
  const int kb = ss_key_bytes(int(kd));
  if (n < 0 || m < 0 || kb == 0 || (order != AK_ASCENDING && order != AK_DESCENDING)) return AK_ERR_INVALID_ARG;
  if (m == 0) return AK_OK;
  auto misaligned = [](const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) != 0; };
  if (!d_x || !d_out || misaligned(d_x, kb) || misaligned(d_out, 8)) return AK_ERR_INVALID_ARG;
  if (n > 0 && (!d_v || misaligned(d_v, kb))) return AK_ERR_INVALID_ARG;
  return ss_dispatch<LAST>(d_v, n, d_x, m, int(kd), order == AK_DESCENDING, d_out,
                           reinterpret_cast<cudaStream_t>(stream));
}

}  // namespace
}  // namespace ak

extern "C" {

ak_status ak_searchsortedfirst(const void *d_v, int64_t n, const void *d_x, int64_t m, ak_dtype kd, ak_order order,
                               int64_t *d_out, ak_stream_t stream) {
  return ak::ss_entry<false>(d_v, n, d_x, m, kd, order, d_out, stream);
}

ak_status ak_searchsortedlast(const void *d_v, int64_t n, const void *d_x, int64_t m, ak_dtype kd, ak_order order,
                              int64_t *d_out, ak_stream_t stream) {
  return ak::ss_entry<true>(d_v, n, d_x, m, kd, order, d_out, stream);
}

}  // extern "C"
