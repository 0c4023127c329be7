// merge.cuh -- merge path: stable merges of sorted runs, for the mid-size sort.
//
// The paper's own local sorter is a merge sort (Sec. II-B, AK merge_sort); for
// arrays a few shared-memory tiles long it beats the radix passes, whose cost
// is launch and latency bound there.  The sort takes tiles of CAP keys sorted in
// shared memory by the segmented kernel (one segment per tile), then
// ceil(log2(tiles)) rounds; round r merges runs of width w = CAP * 2^r pairwise
// from one buffer into the other.
//
// merge_pass_kernel: each CTA produces CH = BLOCK * ITEMS consecutive outputs
// of one pair of runs.  The split of its first and last output between the two
// runs is found along the merge-path diagonal by a warp-cooperative 33-way
// search (global memory); both input pieces are staged in shared memory; each
// thread finds its
// own diagonal there and merges ITEMS outputs; the outputs go back through
// shared memory so the stores are coalesced.  Ties take the left run first, so
// every merge -- and the sort -- is stable.  Order is the radix-key order of
// common.cuh, so Julia isless (and its reverse) holds.
#pragma once

#include "common.cuh"

namespace ak {

// Number of elements of A among the first d outputs of the stable merge of
// A[0, la) and B[0, lb) (A before B on ties).
template <int KIND, typename U>
__device__ __forceinline__ int64_t merge_split(const U *A, int64_t la, const U *B, int64_t lb, int64_t d, U flip) {
  int64_t lo = d - lb > 0 ? d - lb : 0, hi = d < la ? d : la;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (radix_key_t<KIND>(A[mid], flip) <= radix_key_t<KIND>(B[d - 1 - mid], flip)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The same split found by one warp: each round the 32 lanes probe 32 points of
// the candidate range at once (a 33-way search), so a range of 2^k positions
// needs about k / 5 dependent global round trips instead of k.  The predicate
// "A[mid] precedes B[d - 1 - mid]" holds on a prefix of the range.
template <int KIND, typename U>
__device__ __forceinline__ int64_t merge_split_warp(const U *A, int64_t la, const U *B, int64_t lb, int64_t d,
                                                    U flip) {
  const int lane = threadIdx.x & 31;
  int64_t lo = d - lb > 0 ? d - lb : 0, hi = d < la ? d : la;  // answer in [lo, hi]
  auto before = [&](int64_t mid) {
    return radix_key_t<KIND>(A[mid], flip) <= radix_key_t<KIND>(B[d - 1 - mid], flip);
  };
  while (hi - lo > 32) {
    const int64_t span = hi - lo;
    const int64_t p = lo + (span * (lane + 1)) / 33;  // strictly inside [lo, hi)
    const uint32_t t = __ballot_sync(0xffffffffu, before(p));
    const int k = __popc(t);  // the predicate holds on probes 0 .. k-1
    const int64_t plo = __shfl_sync(0xffffffffu, p, k > 0 ? k - 1 : 0);
    const int64_t phi = __shfl_sync(0xffffffffu, p, k < 32 ? k : 31);
    if (k > 0) lo = plo + 1;
    if (k < 32) hi = phi;
  }
  const int64_t q = lo + lane;
  const uint32_t t = __ballot_sync(0xffffffffu, q < hi && before(q));
  return lo + __popc(t);
}

template <typename U, typename V, bool HAS_V, int KIND, int BLOCK, int ITEMS>
__global__ void __launch_bounds__(BLOCK) merge_pass_kernel(const U *__restrict__ sk, const V *__restrict__ sv,
                                                         U *__restrict__ dk, V *__restrict__ dv, int64_t n,
                                                         int64_t w, U flip, int64_t chunks_per_pair,
                                                         int64_t total_chunks) {
  constexpr int CH = BLOCK * ITEMS;
  __shared__ U s_k[CH];
  __shared__ V s_v[HAS_V ? CH : 1];
  __shared__ int64_t s_split[2];
  const int tid = threadIdx.x;
  for (int64_t c = blockIdx.x; c < total_chunks; c += gridDim.x) {
    const int64_t pair = c / chunks_per_pair, local = c % chunks_per_pair;
    const int64_t a0 = pair * 2 * w;
    const int64_t a1 = (a0 + w) < n ? (a0 + w) : n;
    const int64_t b1 = (a0 + 2 * w) < n ? (a0 + 2 * w) : n;
    const int64_t la = a1 - a0, lb = b1 - a1;
    const int64_t o0 = local * CH;
    if (o0 >= la + lb) continue;  // past the end of a short last pair (uniform over the CTA)
    const int64_t o1 = (o0 + CH) < (la + lb) ? (o0 + CH) : (la + lb);
    if (tid < 64) {  // warp 0 splits the first output, warp 1 the end
      const int64_t sp = merge_split_warp<KIND>(sk + a0, la, sk + a1, lb, tid < 32 ? o0 : o1, flip);
      if ((tid & 31) == 0) s_split[tid >> 5] = sp;
    }
    __syncthreads();
    const int64_t ia0 = s_split[0], ia1 = s_split[1];
    const int na = int(ia1 - ia0), nb = int((o1 - ia1) - (o0 - ia0));
    const int64_t ib0 = o0 - ia0;
    for (int i = tid; i < na; i += BLOCK) {
      s_k[i] = sk[a0 + ia0 + i];
      if (HAS_V) s_v[i] = sv[a0 + ia0 + i];
    }
    for (int i = tid; i < nb; i += BLOCK) {
      s_k[na + i] = sk[a1 + ib0 + i];
      if (HAS_V) s_v[na + i] = sv[a1 + ib0 + i];
    }
    __syncthreads();
    const int total = na + nb;
    const int d0 = tid * ITEMS < total ? tid * ITEMS : total;
    int i = int(merge_split<KIND>(s_k, na, s_k + na, nb, d0, flip));
    int j = d0 - i;
    U ok[ITEMS];
    V ov[HAS_V ? ITEMS : 1];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      if (d0 + r < total) {
        const bool take_a = j >= nb || (i < na && radix_key_t<KIND>(s_k[i], flip) <= radix_key_t<KIND>(s_k[na + j], flip));
        const int src = take_a ? i : na + j;
        ok[r] = s_k[src];
        if (HAS_V) ov[r] = s_v[src];
        i += take_a ? 1 : 0;
        j += take_a ? 0 : 1;
      }
    }
    __syncthreads();  // every staged input read
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      if (d0 + r < total) {
        s_k[d0 + r] = ok[r];
        if (HAS_V) s_v[d0 + r] = ov[r];
      }
    }
    __syncthreads();
    for (int q = tid; q < total; q += BLOCK) {
      dk[a0 + o0 + q] = s_k[q];
      if (HAS_V) dv[a0 + o0 + q] = s_v[q];
    }
    __syncthreads();  // the staging buffer is reused by the next chunk
  }
}

}  // namespace ak
