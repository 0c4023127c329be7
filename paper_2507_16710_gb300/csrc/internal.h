// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ak_sort.h"

namespace ak {

struct DevHeader;
struct RadixPlan;
struct LearnedModel;

// One radix sort (keys, keys+values, or keys -> permutation) on device buffers.
struct RadixCall {
  int mode;                // MODE_INPLACE or MODE_PERM
  const void *k_in;        // first pass source
  void *k_final;           // MODE_INPLACE destination (== k_in)
  void *k_alt0, *k_alt1;   // workspace ping-pong (k_alt1 only for MODE_PERM)
  const void *v_in;        // MODE_INPLACE pairs source
  void *v_final;           // pairs destination / permutation output
  void *v_alt;             // workspace ping-pong for values
  int val_bytes;           // 0 = keys only; MODE_PERM uses 4
  int64_t n;
  int kind;                // KeyKind
  int descending;
  int tile_config;         // 0..AK_TILE_CONFIGS-1
  DevHeader *hdr;
  unsigned long long *counts;  // MAX_PASSES * RADIX
  RadixPlan *plan;
  void *status[2];         // look-back words, each num_tiles * RADIX
  uint32_t *chunk_cnt;     // reduce-then-scan passes: RTS_MAX_CHUNKS * RADIX digit counts
  int status_wide;         // 64-bit look-back words (n > 2^30)
  uint64_t timeout_ns;
  int path_tag;            // written to ak_info.path (0 = leave)
  int debug_flags;
  void **pass_events;      // optional profiling events (2 per pass)
  const uint32_t *gate;    // if set, every kernel runs only when *gate == gate_want
  uint32_t gate_want;
  int gather;              // MODE_PERM with keys read through the index (no key copies)
  cudaStream_t stream;
};

// Launch the whole sequence (histogram, plan, passes, finish) on c.stream.
// The header region (status, counters, histogram counts) must be zeroed first.
// One entry point per key word width and key kind (unsigned/signed/float).
cudaError_t radix_launch_u16_uint(const RadixCall &c);
cudaError_t radix_launch_u16_sint(const RadixCall &c);
cudaError_t radix_launch_u16_float(const RadixCall &c);
cudaError_t radix_launch_u16_bf16(const RadixCall &c);
cudaError_t radix_launch_u32_uint(const RadixCall &c);
cudaError_t radix_launch_u32_sint(const RadixCall &c);
cudaError_t radix_launch_u32_float(const RadixCall &c);
cudaError_t radix_launch_u64_uint(const RadixCall &c);
cudaError_t radix_launch_u64_sint(const RadixCall &c);
cudaError_t radix_launch_u64_float(const RadixCall &c);
cudaError_t radix_launch_u128_uint(const RadixCall &c);
cudaError_t radix_launch_u128_sint(const RadixCall &c);

// Tile shapes of the digit-pass kernel.  Configuration c has CFG_BLOCK[c]
// threads and a tile of about CFG_BYTES[c] bytes of keys+values (keys per
// thread clamped to [2, 12]).  Persistent configurations launch one wave of
// CTAs that loop over tiles, each copying its next tile in while it finishes
// the current one; configuration 2 launches one CTA per tile.  Configuration
// 3 is the pass with a dedicated look-back warp (onesweep_ws.cuh): 15 compute
// warps of the 16, keys per thread as many as three tile buffers allow with
// two CTAs per SM.  Configuration 0 (the default) takes 40 KB tiles, the most
// whose stage and digit-order buffers still fit two CTAs per SM for 8-byte
// keys (10 keys per thread): against 32 KB tiles a pass of int64 keys is 9%
// faster, sortperm and 32-bit pairs 10-12%.  Configuration 4 is the
// reduce-then-scan form of configuration 0's tile: an upsweep kernel counts
// each chunk's digits, then one CTA per chunk sorts its consecutive tiles in
// order with running digit offsets and no look-back (onesweep.cuh: RTS).
constexpr int CFG_BLOCK[5] = {512, 384, 512, 512, 512};
constexpr int CFG_BYTES[5] = {40960, 24576, 32768, 0, 40960};
constexpr bool CFG_PERSIST[5] = {true, true, false, true, true};
constexpr int CFG_WS = 3;
constexpr int CFG_RTS = 4;
// Chunks of a reduce-then-scan pass: one per resident CTA, at most this many
// (the workspace holds their digit counts).
constexpr int RTS_MAX_CHUNKS = 1024;
// Configuration of tile_config 0 (the default) and of the learned path's passes.
constexpr int CFG_DEFAULT = 0;

constexpr int WS_BLOCK = 512;       // threads of the look-back-warp pass
constexpr int WS_NCW = 15;          // its compute warps (the last warp looks back)
constexpr int WS_NC = WS_NCW * 32;  // its compute threads
constexpr size_t WS_SMEM_LIMIT = 114 * 1024;  // shared memory per CTA with two CTAs per SM

// Shared memory of the look-back-warp pass (onesweep_ws.cuh: WsSmem): three
// tile buffers, two digit arrays, per-warp digit counters, optional per-warp
// peer words, per-digit state of two tiles.
constexpr size_t ws_smem_bytes(int key_bytes, int val_bytes, int items, bool peer_words) {
  const size_t tile = size_t(WS_NC) * items;
  const size_t buf = (tile * (key_bytes + val_bytes) + 127) / 128 * 128;
  const size_t hist = (size_t(257) * 9 * 4 + 15) / 16 * 16;
  const size_t mask = peer_words ? (size_t(WS_NCW) * 257 * 4 + 15) / 16 * 16 : 0;
  return 3 * buf + (2 * tile + 15) / 16 * 16 + hist + mask + 256 * 8 + 2 * 256 * 4 + 2 * 256 * 8 + 32 + 40 + 16 + 8 +
         16;
}
// Keys per compute thread: its keys, values and digit/rank words stay in
// registers from load to scatter, about 21 registers' worth; and three tile
// buffers fit with two CTAs per SM.
constexpr int ws_items(int key_bytes, int val_bytes, bool peer_words) {
  const int regs = (key_bytes + 3) / 4 + (val_bytes + 3) / 4 + 1;
  int it = 21 / regs < 12 ? 21 / regs : 12;
  if (val_bytes == 0 && key_bytes <= 4 && it > 8) it = 8;  // more spills registers (ptxas -v)
  while (it > 2 && ws_smem_bytes(key_bytes, val_bytes, it, peer_words) > WS_SMEM_LIMIT) --it;
  return it;
}
#ifndef AK_WS_RANK
#define AK_WS_RANK 0
#endif

constexpr int tile_items(int key_bytes, int val_bytes, int cfg) {
  return cfg == CFG_WS ? ws_items(key_bytes, val_bytes, AK_WS_RANK == 1)
         : (CFG_BYTES[cfg] / (CFG_BLOCK[cfg] * (key_bytes + val_bytes))) < 2  ? 2
         : (CFG_BYTES[cfg] / (CFG_BLOCK[cfg] * (key_bytes + val_bytes))) > 12 ? 12
                                                                               : CFG_BYTES[cfg] / (CFG_BLOCK[cfg] * (key_bytes + val_bytes));
}
constexpr int tile_keys(int key_bytes, int val_bytes, int cfg) {
  return (cfg == CFG_WS ? WS_NC : CFG_BLOCK[cfg]) * tile_items(key_bytes, val_bytes, cfg);
}
// 64-bit look-back words (n > 2^30) are built for configurations 0 and 3; the
// reduce-then-scan configuration keeps 32-bit destinations, so above 2^30 keys
// it runs as configuration 0 too.
constexpr int effective_cfg(int cfg, bool status_wide) { return status_wide && cfg != CFG_WS ? 0 : cfg; }

// Keys of one segment the shared-memory sort takes (a multiple of 32): 80 KB
// of keys, values and 16-bit positions, so two CTAs fit an SM.
constexpr int seg_cap(int key_bytes, int val_bytes) { return (81920 / (key_bytes + val_bytes + 2)) / 32 * 32; }

// One segmented sort (or a single segment when off == NULL) on device buffers.
struct SegCall {
  void *keys, *vals;       // in place; vals NULL for keys only
  void *alt_k, *alt_v;     // workspace regions of n elements (segments above the shared capacity)
  int val_bytes;           // 0 = keys only
  const int64_t *off;      // nseg + 1 device offsets, or NULL for one segment [0, n)
  int64_t nseg, n;
  int kind, descending;
  uint32_t *order;         // nseg work-order entries (workspace)
  uint32_t *counters;      // 2 zeroed counters (workspace)
  DevHeader *hdr;          // zeroed header (work counter)
  int path_tag;            // written to ak_info.path
  const uint32_t *gate;    // if set, run only when *gate == gate_want
  uint32_t gate_want;
  int merge;               // off == NULL: sort tiles of the shared-memory capacity, then merge them
  // device-wide split of segments above the shared capacity (segsplit.cuh);
  // all NULL: one CTA sorts such a segment through global memory by itself
  void *split_state;       // SplitState, zeroed
  void *split_big;         // BigSeg[split_big_cap]
  uint32_t *split_tcount;  // RADIX counters per split tile
  void *split_buckets;     // BucketItem[split_bucket_cap]
  int64_t split_min;       // split segments above this many keys; 0: SPLIT_MIN_CAPS x capacity; < 0: none
  cudaStream_t stream;
};
// Split workspace of a segmented sort of n keys (key_bytes + val_bytes wide):
// big segments hold more than the shared capacity each; every one of them
// gets at most 4 len / CAP non-empty buckets (buckets average more than CAP / 4).
constexpr int64_t split_big_cap(int64_t n, int key_bytes, int val_bytes) {
  return n / (int64_t(seg_cap(key_bytes, val_bytes)) + 1) + 1;
}
constexpr int64_t split_bucket_cap(int64_t n, int key_bytes, int val_bytes) {
  return 4 * (n / seg_cap(key_bytes, val_bytes)) + 256;
}
// Segments above SPLIT_MIN_CAPS times the shared capacity are split across all
// CTAs before the per-CTA sort (segsplit.cuh); shorter ones above the capacity
// are taken by one CTA through global memory, overlapped with other work.
constexpr int SPLIT_MIN_CAPS = 8;
// Split tiles: SPLIT_BLOCK threads x up to 8 keys, about 32 KB of keys and values.
constexpr int SPLIT_BLOCK = 512;
constexpr int SPLIT_TILE_BYTES = 32768;
constexpr int split_items(int key_bytes, int val_bytes) {
  return SPLIT_TILE_BYTES / (SPLIT_BLOCK * (key_bytes + val_bytes)) < 1   ? 1
         : SPLIT_TILE_BYTES / (SPLIT_BLOCK * (key_bytes + val_bytes)) > 8 ? 8
                                                                          : SPLIT_TILE_BYTES / (SPLIT_BLOCK * (key_bytes + val_bytes));
}
constexpr int split_tile(int key_bytes, int val_bytes) { return SPLIT_BLOCK * split_items(key_bytes, val_bytes); }
constexpr int64_t split_tile_cap(int64_t n, int key_bytes, int val_bytes) {
  return n / split_tile(key_bytes, val_bytes) + split_big_cap(n, key_bytes, val_bytes) + 1;
}

// Learned-CDF path: model, sample and finish regions of the workspace.
struct LearnedCall {
  LearnedModel *model;         // zeroed
  uint32_t m, seed;            // sample size, sample/initialisation seed
  unsigned long long *sample_r;
  float *xs, *xs_v;            // x-hat of the sorted sample: radix / value coordinate
  RadixCall sample_sort;       // radix sort of sample_r (u64 keys) in place
  float *partials;             // training partial sums
  int train_steps;             // 0: piecewise-linear CDF only
  float lr;
  uint32_t nbuckets, bucket_bits;
  uint32_t *bucket_counts;     // nbuckets, zeroed
  int64_t *seg_off;            // nbuckets + 1 bucket offsets
  int64_t seg_capacity;        // shared-memory capacity of the finish
  uint16_t *ids, *ids_alt;     // keys-only sorts: n bucket ids and their pass copy (else NULL)
  SegCall finish;              // segmented sort over the buckets
};
cudaError_t learned_launch_u16_uint(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u16_sint(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u16_float(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u16_bf16(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u32_uint(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u32_sint(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u32_float(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u64_uint(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u64_sint(const RadixCall &c, const LearnedCall &lc);
cudaError_t learned_launch_u64_float(const RadixCall &c, const LearnedCall &lc);
size_t learned_model_bytes();
size_t learned_partials_bytes();
cudaError_t seg_launch_u16_uint(const SegCall &c);
cudaError_t seg_launch_u16_sint(const SegCall &c);
cudaError_t seg_launch_u16_float(const SegCall &c);
cudaError_t seg_launch_u16_bf16(const SegCall &c);
cudaError_t seg_launch_u32_uint(const SegCall &c);
cudaError_t seg_launch_u32_sint(const SegCall &c);
cudaError_t seg_launch_u32_float(const SegCall &c);
cudaError_t seg_launch_u64_uint(const SegCall &c);
cudaError_t seg_launch_u64_sint(const SegCall &c);
cudaError_t seg_launch_u64_float(const SegCall &c);

int device_sm_count();

// Copies the caller's options (or the defaults) into *o; false when a field is
// out of its documented range.
bool resolve_options(const ak_options *opt, ak_options *o);

// Autotune cache: the tuned path and tile configuration of a call shape.
bool tune_lookup(int op, int dtype, int64_t n, int val_bytes, int *path, int *tile_config, int *bucket_bits);
// Autotune cache of the segmented sort: the split threshold (in capacities,
// -1 = never) of a batch shape.
bool tune_lookup_segmented(int dtype, int64_t n, int64_t nseg, int *split_caps);
// Bucket bits the learned path picks by itself for a call shape.
int learned_auto_bucket_bits(int op, int64_t n, int key_bytes, int val_bytes);

}  // namespace ak
