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
// Two levels, for a latency-bound search on GB300:
//  * a table of K pivot keys in shared memory (16 KB: K = 8192, 4096, 2048 for
//    2-, 4-, 8-byte keys), v at positions P_i = floor(i n / (K + 1)),
//    i = 1..K, loaded once per CTA; the table narrows each query to the stretch
//    (P_c, P_{c+1}] of about n / (K + 1) keys with no global access;
//  * bisection in global memory over that stretch, log2(n / K) dependent loads,
//    the upper ones shared by many queries and held in the 129 MB L2.
// Persistent CTAs (a grid of the resident count) walk the queries, so each CTA
// loads its table once.  Reads of x and writes of out are coalesced.
//
// Bounds: K <= n - 1, so the pivots strictly increase and (P_c, P_{c+1}] stays
// inside [0, n) whatever v holds; an unsorted v gives unspecified answers in
// [0, n] (first) or [-1, n - 1] (last) and no access outside v[0, n).
#include <mutex>

#include "common.cuh"

namespace ak {

constexpr int SS_BLOCK = 512;
constexpr int SS_TABLE_BYTES = 16384;

// floor(i * n / parts) as i * q + floor(i * r / parts), n = q * parts + r:
// exact, and no intermediate exceeds n or parts^2.
__device__ __forceinline__ int64_t ss_pivot(int64_t i, int64_t q, int64_t r, int64_t parts) {
  return i * q + (i * r) / parts;
}

template <typename U, int KIND, bool LAST>
__global__ void __launch_bounds__(SS_BLOCK) searchsorted_kernel(const U *__restrict__ v, int64_t n,
                                                                const U *__restrict__ x, int64_t m, U flip, int K,
                                                                int64_t *__restrict__ out) {
  constexpr int TABLE = SS_TABLE_BYTES / int(sizeof(U));
  __shared__ U s_t[TABLE];
  const int64_t parts = int64_t(K) + 1, q = n / parts, r = n % parts;
  for (int i = threadIdx.x; i < K; i += SS_BLOCK) s_t[i] = radix_key_t<KIND>(v[ss_pivot(i + 1, q, r, parts)], flip);
  __syncthreads();
  const int64_t stride = int64_t(gridDim.x) * SS_BLOCK;
  for (int64_t g = int64_t(blockIdx.x) * SS_BLOCK + threadIdx.x; g < m; g += stride) {
    const U key = radix_key_t<KIND>(x[g], flip);
    // the predicate that holds on a prefix of a sorted v
    auto in_prefix = [key](U e) { return LAST ? e <= key : e < key; };
    int c = 0, len = K;  // c = table entries in the prefix
    while (len > 0) {
      const int half = len >> 1;
      if (in_prefix(s_t[c + half])) {
        c += half + 1;
        len -= half + 1;
      } else {
        len = half;
      }
    }
    // pivot c (table entry c - 1) is in the prefix, pivot c + 1 is not
    int64_t lo = c == 0 ? 0 : ss_pivot(c, q, r, parts) + 1;
    int64_t span = (c == K ? n : ss_pivot(c + 1, q, r, parts)) - lo;
    while (span > 0) {
      const int64_t half = span >> 1;
      if (in_prefix(radix_key_t<KIND>(v[lo + half], flip))) {
        lo += half + 1;
        span -= half + 1;
      } else {
        span = half;
      }
    }
    out[g] = LAST ? lo - 1 : lo;
  }
}

namespace {

// Resident CTAs per SM of one kernel on the current device (cached: the
// occupancy query is a host computation but not free).
int ss_resident_ctas(const void *fn, int dev) {
  static std::mutex mu;
  static const void *fns[64];
  static int devs[64], vals[64], used = 0;
  std::lock_guard<std::mutex> lock(mu);
  for (int i = 0; i < used; ++i)
    if (fns[i] == fn && devs[i] == dev) return vals[i];
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, SS_BLOCK, 0) != cudaSuccess) return 0;
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
  auto *fn = searchsorted_kernel<U, KIND, LAST>;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AK_ERR_CUDA;
  const int resident = ss_resident_ctas(reinterpret_cast<const void *>(fn), dev);
  if (resident <= 0) return AK_ERR_CUDA;
  const int64_t want = (m + SS_BLOCK - 1) / SS_BLOCK;
  const int grid = int(want < resident ? want : resident);
  const int K = int(n - 1 < TABLE ? (n > 0 ? n - 1 : 0) : TABLE);
  const U flip = desc ? U(~U(0)) : U(0);
  fn<<<grid, SS_BLOCK, 0, stream>>>(static_cast<const U *>(v), n, static_cast<const U *>(x), m, flip, K, out);
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
  }
  return AK_ERR_INVALID_ARG;
}

int ss_key_bytes(int kd) {
  switch (kd) {
    case AK_U16: case AK_I16: case AK_F16: case AK_BF16: return 2;
    case AK_U32: case AK_I32: case AK_F32: return 4;
    case AK_U64: case AK_I64: case AK_F64: return 8;
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
