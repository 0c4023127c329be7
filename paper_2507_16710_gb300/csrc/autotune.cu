// autotune.cu -- timed choice of path and tile configuration per call shape.
//
// ak_autotune runs every candidate (radix with each tile configuration -- the
// configurations differ in threads per CTA, keys per thread and persistence --, the
// learned path with its own bucket count and with half and twice as many
// buckets, the one-launch block path when n fits it, else the merge path up to
// 2^26 keys) on the caller's
// buffers, restoring the inputs from a copy in the workspace before each timed
// call, times it with CUDA events on the caller's stream and records the
// fastest under (op, dtype, ceil(log2 n), value bytes).  AK_PATH_AUTO
// calls consult this cache (ak_sort_temp_bytes too, so sizes agree).  The cache
// is kept in host memory behind a mutex and persists as JSON lines.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.h"

namespace ak {
namespace {

struct TuneEntry {
  int path, tile_config, bucket_bits;
  float ms;
  int split_caps;  // segmented entries: split threshold in capacities (-1 = never)
};
using TuneKey = std::tuple<int, int, int, int>;  // op, dtype, log2 n, value bytes

std::mutex g_mu;
std::map<TuneKey, TuneEntry> g_cache;
bool g_env_loaded = false;

int log2_class(int64_t n) {
  int b = 0;
  while ((int64_t(1) << b) < n) ++b;
  return b;
}

ak_status load_file(const char *path) {
  FILE *f = fopen(path, "r");
  if (!f) return AK_ERR_INVALID_ARG;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    int op, dt, lg, vb, pth, tc, bb = 0, sc = 0;
    float ms;
    // bucket_bits and split_caps are optional (absent: "automatic")
    const int got = sscanf(line,
                           " {\"op\": %d, \"dtype\": %d, \"log2n\": %d, \"val_bytes\": %d, \"path\": %d, "
                           "\"tile_config\": %d, \"ms\": %f, \"bucket_bits\": %d, \"split_caps\": %d}",
                           &op, &dt, &lg, &vb, &pth, &tc, &ms, &bb, &sc);
    if ((got >= 7 && got <= 9) && pth >= AK_PATH_RADIX && pth <= AK_PATH_MERGE && tc >= 0 &&
        tc <= AK_TILE_CONFIGS && (bb == 0 || (bb >= 8 && bb <= 16)) && sc >= -1 && sc <= 1024)
      g_cache[TuneKey(op, dt, lg, vb)] = TuneEntry{pth, tc, bb, ms, sc};
  }
  fclose(f);
  return AK_OK;
}

void load_env_once() {  // caller holds g_mu
  if (g_env_loaded) return;
  g_env_loaded = true;
  const char *p = getenv("AK_TUNE_CACHE");
  if (p && *p) load_file(p);
}

}  // namespace

bool tune_lookup(int op, int dtype, int64_t n, int val_bytes, int *path, int *tile_config, int *bucket_bits) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_env_once();
  auto it = g_cache.find(TuneKey(op, dtype, log2_class(n), val_bytes));
  if (it == g_cache.end()) return false;
  *path = it->second.path;
  *tile_config = it->second.tile_config;
  *bucket_bits = it->second.bucket_bits;
  return true;
}

bool tune_lookup_segmented(int dtype, int64_t n, int64_t nseg, int *split_caps) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_env_once();
  auto it = g_cache.find(TuneKey(AK_OP_SORT_SEGMENTED, dtype, log2_class(n), log2_class(nseg)));
  if (it == g_cache.end() || it->second.split_caps == 0) return false;
  *split_caps = it->second.split_caps;
  return true;
}

}  // namespace ak

using namespace ak;

static int key_bytes_of(ak_dtype kd) {
  switch (kd) {
    case AK_U16: case AK_I16: case AK_F16: case AK_BF16: return 2;
    case AK_U32: case AK_I32: case AK_F32: return 4;
    case AK_U64: case AK_I64: case AK_F64: return 8;
    case AK_U128: case AK_I128: return 16;
  }
  return 0;
}

// Candidates of one call shape and the workspace ak_autotune needs for them:
// the largest candidate's temporaries (256-byte aligned), then a copy of the inputs.
static ak_status candidates(int op, int64_t n, ak_dtype kd, int val_bytes, std::vector<ak_options> *cands,
                            size_t *need, size_t *input_bytes) {
  if (op != AK_OP_SORT && op != AK_OP_SORTPERM && op != AK_OP_SORT_PAIRS) return AK_ERR_INVALID_ARG;
  const int kb = key_bytes_of(kd);
  if (n <= 0 || kb == 0) return AK_ERR_INVALID_ARG;
  if (kb == 16) return AK_ERR_UNSUPPORTED;  // 128-bit keys have one configuration: nothing to choose
  const int vb = (op == AK_OP_SORT_PAIRS) ? val_bytes : 0;
  if (op == AK_OP_SORT_PAIRS && vb != 1 && vb != 2 && vb != 4 && vb != 8) return AK_ERR_INVALID_ARG;
  cands->clear();
  for (int tc = 1; tc <= AK_TILE_CONFIGS; ++tc) {
    ak_options o{};
    o.path = AK_PATH_RADIX;
    o.tile_config = tc;
    cands->push_back(o);
  }
  if (n >= (int64_t(1) << 16) && n < (int64_t(1) << 32)) {
    const int bb = learned_auto_bucket_bits(op, n, kb, vb);
    for (int d = -1; d <= 1; ++d) {  // its own bucket count, then half and twice as many buckets
      const int b = d == 0 ? 0 : bb + d;
      if (b != 0 && (b < 8 || b > 16)) continue;
      ak_options o{};
      o.path = AK_PATH_LEARNED;
      o.bucket_bits = b;
      cands->push_back(o);
    }
  }
  if (n <= seg_cap(kb, op == AK_OP_SORTPERM ? 4 : vb)) {
    ak_options o{};
    o.path = AK_PATH_BLOCK;
    cands->push_back(o);
  } else if (n <= (int64_t(1) << 26)) {  // a few tiles to a few thousand: tile sort + merge rounds
    ak_options o{};
    o.path = AK_PATH_MERGE;
    cands->push_back(o);
  }
  size_t m = 0;
  for (const ak_options &o : *cands) {
    size_t b = 0;
    if (ak_sort_temp_bytes(op, n, kd, val_bytes, 0, &o, &b) == AK_OK && b > m) m = b;
  }
  *need = (m + 255) & ~size_t(255);
  *input_bytes = size_t(n) * kb + size_t(n) * vb;
  return AK_OK;
}


extern "C" {

ak_status ak_autotune_temp_bytes(int op, int64_t n, ak_dtype kd, int val_bytes, size_t *bytes) {
  if (!bytes) return AK_ERR_INVALID_ARG;
  std::vector<ak_options> cands;
  size_t need = 0, in = 0;
  const ak_status s = candidates(op, n, kd, val_bytes, &cands, &need, &in);
  if (s != AK_OK) return s;
  *bytes = need + in;
  return AK_OK;
}

ak_status ak_autotune(int op, int64_t n, ak_dtype kd, int val_bytes, ak_order order, void *d_keys, void *d_vals,
                      uint32_t *d_perm, void *d_temp, size_t temp_bytes, ak_stream_t stream, ak_options *best) {
  std::vector<ak_options> cands;
  size_t need = 0, inb = 0;
  const ak_status cs = candidates(op, n, kd, val_bytes, &cands, &need, &inb);
  if (cs != AK_OK) return cs;
  (void)inb;
  if (!d_keys || !d_temp || (op == AK_OP_SORT_PAIRS && !d_vals) || (op == AK_OP_SORTPERM && !d_perm))
    return AK_ERR_INVALID_ARG;
  const int kb = key_bytes_of(kd);
  const int vb = (op == AK_OP_SORT_PAIRS) ? val_bytes : 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t kbytes = size_t(n) * kb, vbytes = size_t(n) * vb;
  if (temp_bytes < need + kbytes + vbytes) return AK_ERR_WORKSPACE_TOO_SMALL;
  uint8_t *copy_k = static_cast<uint8_t *>(d_temp) + need;
  uint8_t *copy_v = copy_k + kbytes;
  if (cudaMemcpyAsync(copy_k, d_keys, kbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return AK_ERR_CUDA;
  if (vbytes && cudaMemcpyAsync(copy_v, d_vals, vbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return AK_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AK_ERR_CUDA;
  }
  ak_status result = AK_OK;
  float best_ms = INFINITY;
  ak_options best_o{};
  for (const ak_options &o : cands) {
    float tot = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {  // one warm-up, three timed
      if (cudaMemcpyAsync(d_keys, copy_k, kbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          (vbytes && cudaMemcpyAsync(d_vals, copy_v, vbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) ||
          cudaEventRecord(e0, st) != cudaSuccess) {
        ok = false;
        break;
      }
      ak_status s = AK_OK;
      if (op == AK_OP_SORT) s = ak_sort(d_keys, n, kd, order, d_temp, need, stream, &o);
      else if (op == AK_OP_SORTPERM) s = ak_sortperm(d_keys, d_perm, n, kd, order, d_temp, need, stream, &o);
      else s = ak_sort_pairs(d_keys, d_vals, val_bytes, n, kd, order, d_temp, need, stream, &o);
      if (s != AK_OK || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        ok = false;
        break;
      }
      if (ak_status_check(d_temp, stream) != AK_OK) ok = false;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;
    }
    if (ok && tot / 3.f < best_ms) {
      best_ms = tot / 3.f;
      best_o = o;
    }
  }
  // leave the inputs as they were
  if (cudaMemcpyAsync(d_keys, copy_k, kbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      (vbytes && cudaMemcpyAsync(d_vals, copy_v, vbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
    result = AK_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) result = AK_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!isfinite(best_ms)) return result == AK_OK ? AK_ERR_CUDA : result;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[TuneKey(op, int(kd), log2_class(n), vb)] = TuneEntry{best_o.path, best_o.tile_config, best_o.bucket_bits,
                                                                 best_ms, 0};
  }
  if (best) *best = best_o;
  return result;
}

static const int kSplitCands[] = {1, 2, 4, 8, 16, -1};

ak_status ak_autotune_segmented_temp_bytes(int64_t n, int64_t nseg, ak_dtype kd, size_t *bytes) {
  if (!bytes || n <= 0 || nseg <= 0 || key_bytes_of(kd) == 0) return AK_ERR_INVALID_ARG;
  size_t need = 0;
  const ak_status s = ak_sort_temp_bytes(AK_OP_SORT_SEGMENTED, n, kd, 0, nseg, nullptr, &need);
  if (s != AK_OK) return s;
  *bytes = ((need + 255) & ~size_t(255)) + size_t(n) * key_bytes_of(kd);
  return AK_OK;
}

ak_status ak_autotune_segmented(void *d_keys, const int64_t *d_offsets, int64_t nseg, int64_t n, ak_dtype kd,
                                ak_order order, void *d_temp, size_t temp_bytes, ak_stream_t stream,
                                ak_options *best) {
  size_t total = 0;
  const ak_status ts = ak_autotune_segmented_temp_bytes(n, nseg, kd, &total);
  if (ts != AK_OK) return ts;
  if (!d_keys || !d_offsets || !d_temp) return AK_ERR_INVALID_ARG;
  if (temp_bytes < total) return AK_ERR_WORKSPACE_TOO_SMALL;
  const size_t kbytes = size_t(n) * key_bytes_of(kd);
  const size_t need = total - kbytes;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint8_t *copy_k = static_cast<uint8_t *>(d_temp) + need;
  if (cudaMemcpyAsync(copy_k, d_keys, kbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return AK_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return AK_ERR_CUDA;
  }
  ak_status result = AK_OK;
  float best_ms = INFINITY;
  int best_caps = 0;
  for (int caps : kSplitCands) {
    ak_options o{};
    o.split_caps = caps;
    float tot = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {  // one warm-up, three timed
      if (cudaMemcpyAsync(d_keys, copy_k, kbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaEventRecord(e0, st) != cudaSuccess) {
        ok = false;
        break;
      }
      const ak_status s = ak_sort_segmented(d_keys, d_offsets, nseg, n, kd, order, d_temp, need, stream, &o);
      if (s != AK_OK || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
        ok = false;
        break;
      }
      if (ak_status_check(d_temp, stream) != AK_OK) ok = false;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;
    }
    if (ok && tot / 3.f < best_ms) {
      best_ms = tot / 3.f;
      best_caps = caps;
    }
  }
  if (cudaMemcpyAsync(d_keys, copy_k, kbytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) result = AK_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) result = AK_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!isfinite(best_ms)) return result == AK_OK ? AK_ERR_CUDA : result;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[TuneKey(AK_OP_SORT_SEGMENTED, int(kd), log2_class(n), log2_class(nseg))] =
        TuneEntry{AK_PATH_BLOCK, 0, 0, best_ms, best_caps};
  }
  if (best) {
    *best = ak_options{};
    best->split_caps = best_caps;
  }
  return result;
}

ak_status ak_autotune_save(const char *path) {
  if (!path) return AK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  FILE *f = fopen(path, "w");
  if (!f) return AK_ERR_INVALID_ARG;
  for (const auto &kv : g_cache) {
    int op, dt, lg, vb;
    std::tie(op, dt, lg, vb) = kv.first;
    fprintf(f,
            "{\"op\": %d, \"dtype\": %d, \"log2n\": %d, \"val_bytes\": %d, \"path\": %d, "
            "\"tile_config\": %d, \"ms\": %.6f, \"bucket_bits\": %d, \"split_caps\": %d}\n",
            op, dt, lg, vb, kv.second.path, kv.second.tile_config, kv.second.ms, kv.second.bucket_bits,
            kv.second.split_caps);
  }
  fclose(f);
  return AK_OK;
}

ak_status ak_autotune_load(const char *path) {
  if (!path) return AK_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  return load_file(path);
}

void ak_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache.clear();
  g_env_loaded = true;  // an explicit clear also drops the environment's cache
}

}  // extern "C"
