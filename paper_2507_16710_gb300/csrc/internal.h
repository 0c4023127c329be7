// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/ak_sort.h"

namespace ak {

struct DevHeader;
struct RadixPlan;

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
  int status_wide;         // 64-bit look-back words (n > 2^30)
  uint64_t timeout_ns;
  int path_tag;            // written to ak_info.path (0 = leave)
  int debug_flags;
  void **pass_events;      // optional profiling events (2 per pass)
  cudaStream_t stream;
};

// Launch the whole sequence (histogram, plan, passes, finish) on c.stream.
// The header region (status, counters, histogram counts) must be zeroed first.
cudaError_t radix_launch_u16(const RadixCall &c);
cudaError_t radix_launch_u32(const RadixCall &c);
cudaError_t radix_launch_u64(const RadixCall &c);

// Keys per tile of a tile configuration (for workspace sizing).
int radix_tile_keys(int key_bytes, int tile_config);
int radix_min_tile_keys(int key_bytes);

int device_sm_count();

}  // namespace ak
