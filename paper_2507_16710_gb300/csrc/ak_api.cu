// ak_api.cu -- the C ABI: argument checks, workspace layout, path choice and the
// launch sequence on the caller's stream.  No allocation, no stream sync.
#include <string.h>

#include <type_traits>

#include <atomic>

#include "internal.h"
#include "learned.cuh"
#include "onesweep.cuh"

namespace ak {

int device_sm_count() {
  static std::atomic<int> cache[64];  // zero-initialised (static storage); one value per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  if (dev >= 0 && dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  if (dev >= 0 && dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

// Smallest tile of any configuration for these widths (sizes the look-back
// arrays so that every configuration fits).
static int min_tile_keys(int key_bytes, int val_bytes) {
  int m = tile_keys(key_bytes, val_bytes, 0);
  for (int c = 1; c < AK_TILE_CONFIGS; ++c) m = m < tile_keys(key_bytes, val_bytes, c) ? m : tile_keys(key_bytes, val_bytes, c);
  return m;
}

static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct KeyInfo {
  int bytes;
  int kind;
};

static bool key_info(int kd, KeyInfo *ki) {
  switch (kd) {
    case AK_U16: *ki = {2, KIND_UINT}; return true;
    case AK_I16: *ki = {2, KIND_SINT}; return true;
    case AK_U32: *ki = {4, KIND_UINT}; return true;
    case AK_I32: *ki = {4, KIND_SINT}; return true;
    case AK_U64: *ki = {8, KIND_UINT}; return true;
    case AK_I64: *ki = {8, KIND_SINT}; return true;
    case AK_F32: *ki = {4, KIND_FLOAT}; return true;
    case AK_F64: *ki = {8, KIND_FLOAT}; return true;
    case AK_F16: *ki = {2, KIND_FLOAT}; return true;
    case AK_BF16: *ki = {2, KIND_BF16}; return true;
    case AK_U128: *ki = {16, KIND_UINT}; return true;
    case AK_I128: *ki = {16, KIND_SINT}; return true;
  }
  return false;
}

// 128-bit keys take the radix path only (AUTO resolves to it).
static bool path_supported(const KeyInfo &ki, const ak_options &o) {
  return ki.bytes != 16 || o.path == AK_PATH_AUTO || o.path == AK_PATH_RADIX;
}

// Workspace of the radix path.
struct RadixLayout {
  size_t hdr, counts, plan, status0, status1, chunk, k_alt0, k_alt1, v_alt, total;
  int status_wide;
};

static RadixLayout radix_layout(int op, int64_t n, int key_bytes, int val_bytes, int tile_keys) {
  RadixLayout L{};
  size_t off = 0;
  L.hdr = off;
  off += align256(sizeof(DevHeader));
  L.counts = off;
  off += align256(sizeof(unsigned long long) * MAX_PASSES * RADIX);
  L.plan = off;
  off += align256(sizeof(RadixPlan));
  const int64_t tiles = (n + tile_keys - 1) / tile_keys;
  // A pass that moves data has every digit count below n, so 30-bit look-back
  // counts hold any n <= 2^30.
  L.status_wide = n > (int64_t(1) << 30);
  const size_t sw = L.status_wide ? 8 : 4;
  L.status0 = off;
  off += align256(size_t(tiles) * RADIX * sw);
  L.status1 = off;
  off += align256(size_t(tiles) * RADIX * sw);
  if (op != AK_OP_SORTPERM_LOWMEM) {  // digit counts per chunk of the reduce-then-scan configuration
    L.chunk = off;
    off += align256(size_t(tiles < RTS_MAX_CHUNKS ? tiles : RTS_MAX_CHUNKS) * RADIX * 4);
  }
  if (op != AK_OP_SORTPERM_LOWMEM) {  // the low-memory sortperm keeps no key copy
    L.k_alt0 = off;
    off += align256(size_t(n) * key_bytes);
  }
  if (op == AK_OP_SORTPERM) {
    L.k_alt1 = off;
    off += align256(size_t(n) * key_bytes);
    L.v_alt = off;
    off += align256(size_t(n) * 4);
  } else if (op == AK_OP_SORTPERM_LOWMEM) {
    L.v_alt = off;
    off += align256(size_t(n) * 4);
  } else if (op == AK_OP_SORT_PAIRS) {
    L.v_alt = off;
    off += align256(size_t(n) * val_bytes);
  }
  L.total = off;
  return L;
}

// Copies the caller's options (or the defaults) into *o; false when a field is
// out of its documented range.
bool resolve_options(const ak_options *opt, ak_options *o) {
  *o = ak_options{};
  if (opt) *o = *opt;
  if (o->path < AK_PATH_AUTO || o->path > AK_PATH_MERGE) return false;
  if (o->tile_config < 0 || o->tile_config > AK_TILE_CONFIGS) return false;
  if (o->bucket_bits != 0 && (o->bucket_bits < 8 || o->bucket_bits > 16)) return false;
  if (o->train_steps < -1) return false;
  if (o->debug_flags & ~(AK_DEBUG_SKIP_FIRST_TILE | AK_DEBUG_NO_PREFETCH | AK_DEBUG_NO_PACK)) return false;
  if (o->digit_bits != 0 && o->digit_bits != RADIX_BITS) return false;
  if (o->split_caps < -1 || o->split_caps > 1024) return false;
  for (int r : o->reserved)
    if (r != 0) return false;
  if (o->timeout_ns == 0) o->timeout_ns = 1000000000ull;
  return true;
}

// AK_PATH_AUTO with no explicit tile configuration takes the autotuned choice.
static void apply_tuning(int op, int kd, int64_t n, int val_bytes, ak_options &o) {
  if (o.path != AK_PATH_AUTO || o.tile_config != 0) return;
  int path = 0, tc = 0, bb = 0;
  if (tune_lookup(op, kd, n, op == AK_OP_SORT_PAIRS ? val_bytes : 0, &path, &tc, &bb)) {
    o.path = path;
    o.tile_config = tc;
    if (o.bucket_bits == 0) o.bucket_bits = bb;
  }
}

static cudaError_t radix_dispatch(int key_bytes, const RadixCall &c) {
  switch (key_bytes) {
    case 2:
      return c.kind == KIND_BF16    ? radix_launch_u16_bf16(c)
             : c.kind == KIND_FLOAT ? radix_launch_u16_float(c)
             : c.kind == KIND_SINT  ? radix_launch_u16_sint(c)
                                    : radix_launch_u16_uint(c);
    case 4:
      return c.kind == KIND_FLOAT  ? radix_launch_u32_float(c)
             : c.kind == KIND_SINT ? radix_launch_u32_sint(c)
                                   : radix_launch_u32_uint(c);
    case 16:
      return c.kind == KIND_SINT ? radix_launch_u128_sint(c) : radix_launch_u128_uint(c);
    default:
      return c.kind == KIND_FLOAT  ? radix_launch_u64_float(c)
             : c.kind == KIND_SINT ? radix_launch_u64_sint(c)
                                   : radix_launch_u64_uint(c);
  }
}

static cudaError_t seg_dispatch(int key_bytes, const SegCall &c) {
  switch (key_bytes) {
    case 2:
      return c.kind == KIND_BF16    ? seg_launch_u16_bf16(c)
             : c.kind == KIND_FLOAT ? seg_launch_u16_float(c)
             : c.kind == KIND_SINT  ? seg_launch_u16_sint(c)
                                    : seg_launch_u16_uint(c);
    case 4:
      return c.kind == KIND_FLOAT  ? seg_launch_u32_float(c)
             : c.kind == KIND_SINT ? seg_launch_u32_sint(c)
                                   : seg_launch_u32_uint(c);
    default:
      return c.kind == KIND_FLOAT  ? seg_launch_u64_float(c)
             : c.kind == KIND_SINT ? seg_launch_u64_sint(c)
                                   : seg_launch_u64_uint(c);
  }
}

// Workspace of the segmented / one-launch block path.
struct SegLayout {
  size_t hdr, counters, split_state, order, alt_k, alt_v, key_copy, split_big, split_tcount, split_buckets, total;
};

static SegLayout seg_layout(int op, int64_t n, int64_t nseg, int key_bytes, int vb) {
  SegLayout L{};
  size_t off = 0;
  L.hdr = off;
  off += align256(sizeof(DevHeader));
  L.counters = off;
  off += 256;
  L.split_state = off;  // zeroed with the header
  off += 256;
  L.order = off;
  off += align256(size_t(nseg > 0 ? nseg : 1) * 4);
  // segments above the shared capacity use a workspace copy
  L.alt_k = off;
  off += align256(size_t(n) * key_bytes);
  L.alt_v = off;
  off += align256(size_t(n) * vb);
  if (op == AK_OP_SORTPERM) {  // the keys are read-only: sort a copy
    L.key_copy = off;
    off += align256(size_t(n) * key_bytes);
  }
  if (op == AK_OP_SORT_SEGMENTED) {  // device-wide split of segments above the shared capacity
    L.split_big = off;
    off += align256(size_t(split_big_cap(n, key_bytes, vb)) * 32);
    L.split_tcount = off;
    off += align256(size_t(split_tile_cap(n, key_bytes, vb)) * RADIX * 4);
    L.split_buckets = off;
    off += align256(size_t(split_bucket_cap(n, key_bytes, vb)) * 16);
  }
  L.total = off;
  return L;
}

__global__ void iota_u32_kernel(uint32_t *p, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = uint32_t(i);
}

// Which path serves a sort/sortperm/pairs call.
// AUTO: one CTA for what fits it; up to eight such tiles, the merge path; learned buckets for large arrays of 64-bit
// keys (2 bucket passes and a shared-memory finish instead of up to 8 radix
// passes, with the on-device fallback for keys the model cannot spread),
// except the sortperm of up to 2^30 of them, whose packed radix passes are
// faster (268M int64 keys: 14.8 ms radix, 15.7 ms learned); radix otherwise.
constexpr int64_t LEARNED_AUTO_MIN = int64_t(1) << 25;
static int choose_path(int op, int64_t n, int key_bytes, int vb, const ak_options &o) {
  if (key_bytes == 16) return AK_PATH_RADIX;
  if (o.path == AK_PATH_RADIX || o.path == AK_PATH_BLOCK || o.path == AK_PATH_MERGE) return o.path;
  if (o.path == AK_PATH_LEARNED) return n < (int64_t(1) << 32) ? AK_PATH_LEARNED : AK_PATH_RADIX;
  if (n <= seg_cap(key_bytes, vb)) return AK_PATH_BLOCK;
  // a few tiles: tile sort + up to three merge rounds beat the radix launches
  // (float64 100K keys 96 vs 112 us; u32 32K 57 vs 71 us)
  if (n <= 8 * int64_t(seg_cap(key_bytes, vb))) return AK_PATH_MERGE;
  if (key_bytes == 8 && op == AK_OP_SORTPERM && n <= (int64_t(1) << 30)) return AK_PATH_RADIX;
  if (key_bytes == 8 && n >= LEARNED_AUTO_MIN && n < (int64_t(1) << 32)) return AK_PATH_LEARNED;
  return AK_PATH_RADIX;
}

static int value_bytes(int op, int val_bytes) {
  return (op == AK_OP_SORTPERM || op == AK_OP_SORTPERM_LOWMEM) ? 4 : (op == AK_OP_SORT_PAIRS ? val_bytes : 0);
}

struct LearnedLayout;
static size_t learned_total(int op, int64_t n, int key_bytes, int val_bytes, const ak_options &o);

static size_t temp_for(int op, int64_t n, int key_bytes, int val_bytes, int64_t nseg, const ak_options &o) {
  const int vb = value_bytes(op, val_bytes);
  if (op == AK_OP_SORT_SEGMENTED) return seg_layout(op, n, nseg, key_bytes, 0).total;
  if (op == AK_OP_SORTPERM_LOWMEM) return radix_layout(op, n, key_bytes, 4, min_tile_keys(key_bytes, 4)).total;
  const int path = choose_path(op, n, key_bytes, vb, o);
  if (path == AK_PATH_BLOCK || path == AK_PATH_MERGE) return seg_layout(op, n, 1, key_bytes, vb).total;
  if (path == AK_PATH_LEARNED) return learned_total(op, n, key_bytes, val_bytes, o);
  return radix_layout(op, n, key_bytes, val_bytes, min_tile_keys(key_bytes, vb)).total;
}

// Segmented sort, or the one-launch block sort of a single segment (off NULL).
static ak_status run_seg(int op, void *keys, const int64_t *off, int64_t nseg, int64_t n, const void *k_in,
                         void *vals, int val_bytes, const KeyInfo &ki, int order, void *d_temp, size_t temp_bytes,
                         cudaStream_t stream, int merge = 0, int64_t split_min = 0) {
  const int vb = value_bytes(op, val_bytes);
  const SegLayout L = seg_layout(op, n, off ? nseg : 1, ki.bytes, vb);
  if (d_temp == nullptr || temp_bytes < L.total) return AK_ERR_WORKSPACE_TOO_SMALL;
  uint8_t *t = static_cast<uint8_t *>(d_temp);
  if (cudaMemsetAsync(t, 0, L.order, stream) != cudaSuccess) return AK_ERR_CUDA;
  void *sort_keys = keys;
  if (op == AK_OP_SORTPERM) {
    sort_keys = t + L.key_copy;
    if (cudaMemcpyAsync(sort_keys, k_in, size_t(n) * ki.bytes, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
      return AK_ERR_CUDA;
    const int g = int((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    iota_u32_kernel<<<g, 256, 0, stream>>>(static_cast<uint32_t *>(vals), n);
  }
  SegCall c{};
  c.keys = sort_keys;
  c.vals = vals;
  c.alt_k = t + L.alt_k;
  c.alt_v = t + L.alt_v;
  c.val_bytes = vb;
  c.off = off;
  c.nseg = off ? nseg : 1;
  c.n = n;
  c.kind = ki.kind;
  c.descending = order == AK_DESCENDING;
  c.order = reinterpret_cast<uint32_t *>(t + L.order);
  c.counters = reinterpret_cast<uint32_t *>(t + L.counters);
  c.hdr = reinterpret_cast<DevHeader *>(t + L.hdr);
  c.path_tag = merge ? AK_PATH_MERGE : AK_PATH_BLOCK;
  c.merge = merge;
  if (op == AK_OP_SORT_SEGMENTED) {
    c.split_min = split_min;
    c.split_state = t + L.split_state;
    c.split_big = t + L.split_big;
    c.split_tcount = reinterpret_cast<uint32_t *>(t + L.split_tcount);
    c.split_buckets = t + L.split_buckets;
  }
  c.stream = stream;
  return seg_dispatch(ki.bytes, c) == cudaSuccess ? AK_OK : AK_ERR_CUDA;
}

// ------------------------------------------------------------ learned path
struct LearnedLayout {
  RadixLayout rad;  // the pairs/keys radix layout (fallback + bucket passes)
  size_t model, sample_r, sample_alt, xs, xs_v, s_hdr, s_counts, s_plan, s_status0, s_status1, partials, bcounts, seg_off,
      seg_order, seg_counters, kcopy, ids, ids_alt, total;
  uint32_t m, bbits;
};

static int ceil_log2(uint64_t v) {
  int b = 0;
  while ((uint64_t(1) << b) < v) ++b;
  return b;
}

static LearnedLayout learned_layout(int op, int64_t n, int key_bytes, int val_bytes, const ak_options &o) {
  LearnedLayout L{};
  // sortperm runs as a key-value sort of a key copy with the index as value
  const int lop = (op == AK_OP_SORTPERM) ? AK_OP_SORT_PAIRS : op;
  const int lvb = (op == AK_OP_SORTPERM) ? 4 : val_bytes;
  const int vb = value_bytes(lop, lvb);
  L.rad = radix_layout(lop, n, key_bytes, lvb, min_tile_keys(key_bytes, vb));
  size_t off = L.rad.total;
  // a 1% sample (at least 4096 keys, at most 2^20)
  int64_t m = n / 100;
  m = m < 4096 ? 4096 : m;
  m = m > LM_MAX_SAMPLE ? LM_MAX_SAMPLE : m;
  m = m > n ? n : m;
  L.m = uint32_t(m);
  // buckets: about half the finish's shared-memory capacity each, 2^8 .. 2^16
  const int64_t per = seg_cap(key_bytes, vb) / 2;
  int bb = (o.bucket_bits >= 8 && o.bucket_bits <= 16) ? o.bucket_bits : ceil_log2(uint64_t((n + per - 1) / per));
  bb = bb < 8 ? 8 : (bb > 16 ? 16 : bb);
  L.bbits = uint32_t(bb);
  const size_t nb = size_t(1) << bb;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += align256(bytes);
    return at;
  };
  L.model = take(sizeof(LearnedModel));
  L.sample_r = take(size_t(m) * 8);
  L.sample_alt = take(size_t(m) * 8);
  L.xs = take(size_t(m) * 4);
  L.xs_v = take(size_t(m) * 4);
  L.s_hdr = take(sizeof(DevHeader));
  L.s_counts = take(sizeof(unsigned long long) * MAX_PASSES * RADIX);
  L.s_plan = take(sizeof(RadixPlan));
  const int64_t stiles = (m + min_tile_keys(8, 0) - 1) / min_tile_keys(8, 0);
  L.s_status0 = take(size_t(stiles) * RADIX * 4);
  L.s_status1 = take(size_t(stiles) * RADIX * 4);
  L.partials = take(learned_partials_bytes());
  L.bcounts = take(nb * 4);
  L.seg_off = take((nb + 1) * 8);
  L.seg_order = take(nb * 4);
  L.seg_counters = take(256);
  if (op == AK_OP_SORTPERM) L.kcopy = take(size_t(n) * key_bytes);
  if (op == AK_OP_SORT) {  // bucket ids carried through the passes as 16-bit values
    L.ids = take(size_t(n) * 2);
    L.ids_alt = take(size_t(n) * 2);
  }
  L.total = off;
  return L;
}

static size_t learned_total(int op, int64_t n, int key_bytes, int val_bytes, const ak_options &o) {
  return learned_layout(op, n, key_bytes, val_bytes, o).total;
}

// Bucket bits the learned path picks by itself for this call shape.
int learned_auto_bucket_bits(int op, int64_t n, int key_bytes, int val_bytes) {
  ak_options o{};
  return int(learned_layout(op, n, key_bytes, val_bytes, o).bbits);
}

static cudaError_t learned_dispatch(int key_bytes, int kind, const RadixCall &c, const LearnedCall &lc) {
  switch (key_bytes) {
    case 2:
      return kind == KIND_BF16    ? learned_launch_u16_bf16(c, lc)
             : kind == KIND_FLOAT ? learned_launch_u16_float(c, lc)
             : kind == KIND_SINT  ? learned_launch_u16_sint(c, lc)
                                  : learned_launch_u16_uint(c, lc);
    case 4:
      return kind == KIND_FLOAT  ? learned_launch_u32_float(c, lc)
             : kind == KIND_SINT ? learned_launch_u32_sint(c, lc)
                                 : learned_launch_u32_uint(c, lc);
    default:
      return kind == KIND_FLOAT  ? learned_launch_u64_float(c, lc)
             : kind == KIND_SINT ? learned_launch_u64_sint(c, lc)
                                 : learned_launch_u64_uint(c, lc);
  }
}

static ak_status run_learned(int op, void *keys, const void *k_in, void *vals, int val_bytes, int64_t n,
                             const KeyInfo &ki, int order, void *d_temp, size_t temp_bytes, cudaStream_t stream,
                             const ak_options &o) {
  const LearnedLayout L = learned_layout(op, n, ki.bytes, val_bytes, o);
  if (d_temp == nullptr || temp_bytes < L.total) return AK_ERR_WORKSPACE_TOO_SMALL;
  uint8_t *t = static_cast<uint8_t *>(d_temp);
  const size_t nb = size_t(1) << L.bbits;
  if (cudaMemsetAsync(t, 0, L.rad.plan, stream) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaMemsetAsync(t + L.model, 0, sizeof(LearnedModel), stream) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaMemsetAsync(t + L.s_hdr, 0, L.s_plan - L.s_hdr, stream) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaMemsetAsync(t + L.bcounts, 0, nb * 4, stream) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaMemsetAsync(t + L.seg_counters, 0, 256, stream) != cudaSuccess) return AK_ERR_CUDA;
  void *kf = keys;
  int vb = val_bytes;
  if (op == AK_OP_SORTPERM) {  // key-value sort of a copy of the keys, values = 0..n-1
    kf = t + L.kcopy;
    if (cudaMemcpyAsync(kf, k_in, size_t(n) * ki.bytes, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
      return AK_ERR_CUDA;
    const int g = int((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    iota_u32_kernel<<<g, 256, 0, stream>>>(static_cast<uint32_t *>(vals), n);
    vb = 4;
  }
  if (op == AK_OP_SORT) vb = 0;
  LearnedModel *md = reinterpret_cast<LearnedModel *>(t + L.model);
  RadixCall c{};
  c.mode = MODE_INPLACE;
  c.k_in = kf;
  c.k_final = kf;
  c.k_alt0 = t + L.rad.k_alt0;
  c.v_in = vals;
  c.v_final = vals;
  c.v_alt = L.rad.v_alt ? t + L.rad.v_alt : nullptr;
  c.val_bytes = vb;
  c.n = n;
  c.kind = ki.kind;
  c.descending = order == AK_DESCENDING;
  c.tile_config = 0;
  c.hdr = reinterpret_cast<DevHeader *>(t + L.rad.hdr);
  c.counts = reinterpret_cast<unsigned long long *>(t + L.rad.counts);
  c.plan = reinterpret_cast<RadixPlan *>(t + L.rad.plan);
  c.status[0] = t + L.rad.status0;
  c.status[1] = t + L.rad.status1;
  c.status_wide = L.rad.status_wide;
  c.timeout_ns = o.timeout_ns;
  c.path_tag = 0;
  c.stream = stream;
  LearnedCall lc{};
  lc.model = md;
  lc.m = L.m;
  lc.seed = o.seed ? o.seed : 0x2507u;
  lc.sample_r = reinterpret_cast<unsigned long long *>(t + L.sample_r);
  lc.xs = reinterpret_cast<float *>(t + L.xs);
  lc.xs_v = reinterpret_cast<float *>(t + L.xs_v);
  RadixCall &sc = lc.sample_sort;
  sc.mode = MODE_INPLACE;
  sc.k_in = lc.sample_r;
  sc.k_final = lc.sample_r;
  sc.k_alt0 = t + L.sample_alt;
  sc.n = L.m;
  sc.kind = KIND_UINT;
  sc.hdr = reinterpret_cast<DevHeader *>(t + L.s_hdr);
  sc.counts = reinterpret_cast<unsigned long long *>(t + L.s_counts);
  sc.plan = reinterpret_cast<RadixPlan *>(t + L.s_plan);
  sc.status[0] = t + L.s_status0;
  sc.status[1] = t + L.s_status1;
  sc.timeout_ns = o.timeout_ns;
  sc.stream = stream;
  lc.partials = reinterpret_cast<float *>(t + L.partials);
  lc.train_steps = o.train_steps < 0 ? 0 : (o.train_steps > 0 ? o.train_steps : 16);
  lc.lr = 1e-2f;
  lc.nbuckets = uint32_t(nb);
  lc.bucket_bits = L.bbits;
  lc.bucket_counts = reinterpret_cast<uint32_t *>(t + L.bcounts);
  lc.seg_off = reinterpret_cast<int64_t *>(t + L.seg_off);
  lc.seg_capacity = seg_cap(ki.bytes, vb);
  lc.ids = L.ids ? reinterpret_cast<uint16_t *>(t + L.ids) : nullptr;
  lc.ids_alt = L.ids_alt ? reinterpret_cast<uint16_t *>(t + L.ids_alt) : nullptr;
  SegCall &f = lc.finish;
  f.keys = kf;
  f.vals = vals;
  f.alt_k = t + L.rad.k_alt0;
  f.alt_v = L.rad.v_alt ? t + L.rad.v_alt : nullptr;
  f.val_bytes = vb;
  f.off = lc.seg_off;
  f.nseg = int64_t(nb);
  f.n = n;
  f.kind = ki.kind;
  f.descending = order == AK_DESCENDING;
  f.order = reinterpret_cast<uint32_t *>(t + L.seg_order);
  f.counters = reinterpret_cast<uint32_t *>(t + L.seg_counters);
  f.hdr = c.hdr;
  f.path_tag = 0;
  f.gate = &md->use_plain;
  f.gate_want = 0;
  f.stream = stream;
  return learned_dispatch(ki.bytes, ki.kind, c, lc) == cudaSuccess ? AK_OK : AK_ERR_CUDA;
}

static bool valid_order(int order) { return order == AK_ASCENDING || order == AK_DESCENDING; }

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Shared tail of sort / sortperm / pairs on the radix path.
static ak_status run_radix(int op, const void *k_in, void *k_final, const void *v_in, void *v_final,
                           int val_bytes, int64_t n, const KeyInfo &ki, int order, void *d_temp,
                           size_t temp_bytes, cudaStream_t stream, const ak_options &o) {
  // Look-back arrays are sized for the smallest tile of any configuration, so
  // every configuration the launcher may pick fits.
  const int vb = value_bytes(op, val_bytes);
  const RadixLayout L = radix_layout(op, n, ki.bytes, val_bytes, min_tile_keys(ki.bytes, vb));
  if (d_temp == nullptr || temp_bytes < L.total) return AK_ERR_WORKSPACE_TOO_SMALL;
  uint8_t *t = static_cast<uint8_t *>(d_temp);
  if (cudaMemsetAsync(t, 0, L.plan, stream) != cudaSuccess) return AK_ERR_CUDA;
  RadixCall c{};
  const bool lowmem = op == AK_OP_SORTPERM_LOWMEM;
  c.mode = (op == AK_OP_SORTPERM || lowmem) ? MODE_PERM : MODE_INPLACE;
  c.gather = lowmem ? 1 : 0;
  c.k_in = k_in;
  c.k_final = k_final;
  c.k_alt0 = lowmem ? nullptr : t + L.k_alt0;
  c.k_alt1 = (op == AK_OP_SORTPERM) ? t + L.k_alt1 : nullptr;
  c.v_in = v_in;
  c.v_final = v_final;
  c.v_alt = L.v_alt ? t + L.v_alt : nullptr;
  c.val_bytes = vb;
  c.n = n;
  c.kind = ki.kind;
  c.descending = order == AK_DESCENDING;
  c.tile_config = (o.tile_config >= 1 && o.tile_config <= AK_TILE_CONFIGS) ? o.tile_config - 1 : CFG_DEFAULT;
  if (lowmem && (c.tile_config == CFG_WS || c.tile_config == CFG_RTS)) c.tile_config = 0;
  c.hdr = reinterpret_cast<DevHeader *>(t + L.hdr);
  c.counts = reinterpret_cast<unsigned long long *>(t + L.counts);
  c.plan = reinterpret_cast<RadixPlan *>(t + L.plan);
  c.status[0] = t + L.status0;
  c.status[1] = t + L.status1;
  c.chunk_cnt = lowmem ? nullptr : reinterpret_cast<uint32_t *>(t + L.chunk);
  c.status_wide = L.status_wide;
  c.timeout_ns = o.timeout_ns;
  c.path_tag = AK_PATH_RADIX;
  c.debug_flags = o.debug_flags;
  c.pass_events = o.pass_events;
  c.stream = stream;
  return radix_dispatch(ki.bytes, c) == cudaSuccess ? AK_OK : AK_ERR_CUDA;
}

}  // namespace ak

using namespace ak;

extern "C" {

const char *ak_version(void) { return "ak_sort 0.1 (sm_103a)"; }

int64_t ak_segment_capacity(int key_bytes, int val_bytes) {
  if (key_bytes != 2 && key_bytes != 4 && key_bytes != 8) return 0;
  if (val_bytes != 0 && val_bytes != 1 && val_bytes != 2 && val_bytes != 4 && val_bytes != 8) return 0;
  return seg_cap(key_bytes, val_bytes);
}

const char *ak_status_string(ak_status s) {
  switch (s) {
    case AK_OK: return "ok";
    case AK_ERR_INVALID_ARG: return "invalid argument";
    case AK_ERR_UNSUPPORTED: return "unsupported request";
    case AK_ERR_WORKSPACE_TOO_SMALL: return "workspace missing or too small";
    case AK_ERR_CUDA: return "CUDA error";
    case AK_ERR_TIMEOUT: return "device-side wait timed out";
    case AK_ERR_INDEX_OVERFLOW: return "n too large for UInt32 indices";
  }
  return "unknown status";
}

ak_status ak_sort_temp_bytes(int op, int64_t n, ak_dtype kd, int val_bytes, int64_t nseg,
                             const ak_options *opt, size_t *bytes) {
  KeyInfo ki;
  if (!bytes || n < 0 || !key_info(kd, &ki)) return AK_ERR_INVALID_ARG;
  if (op < AK_OP_SORT || op > AK_OP_SORTPERM_LOWMEM) return AK_ERR_INVALID_ARG;
  if (op == AK_OP_SORT_PAIRS && val_bytes != 1 && val_bytes != 2 && val_bytes != 4 && val_bytes != 8)
    return AK_ERR_INVALID_ARG;
  if (op == AK_OP_SORT_SEGMENTED && nseg < 0) return AK_ERR_INVALID_ARG;
  ak_options o;
  if (!resolve_options(opt, &o)) return AK_ERR_INVALID_ARG;
  if (ki.bytes == 16 && (op == AK_OP_SORT_SEGMENTED || !path_supported(ki, o))) return AK_ERR_UNSUPPORTED;
  if (op != AK_OP_SORT_SEGMENTED && op != AK_OP_SORTPERM_LOWMEM) apply_tuning(op, kd, n, val_bytes, o);
  *bytes = temp_for(op, n, ki.bytes, val_bytes, nseg, o);
  return AK_OK;
}

ak_status ak_sort(void *d_keys, int64_t n, ak_dtype kd, ak_order order, void *d_temp, size_t temp_bytes,
                  ak_stream_t stream, const ak_options *opt) {
  KeyInfo ki;
  ak_options o;
  if (n < 0 || !key_info(kd, &ki) || !valid_order(order) || !resolve_options(opt, &o)) return AK_ERR_INVALID_ARG;
  if (!path_supported(ki, o)) return AK_ERR_UNSUPPORTED;
  if (n == 0) return AK_OK;
  if (!d_keys || !aligned(d_keys, ki.bytes)) return AK_ERR_INVALID_ARG;
  if (d_temp && !aligned(d_temp, 256)) return AK_ERR_INVALID_ARG;
  apply_tuning(AK_OP_SORT, kd, n, 0, o);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int path = choose_path(AK_OP_SORT, n, ki.bytes, 0, o);
  if (path == AK_PATH_BLOCK || path == AK_PATH_MERGE)
    return run_seg(AK_OP_SORT, d_keys, nullptr, 1, n, nullptr, nullptr, 0, ki, order, d_temp, temp_bytes, st,
                   path == AK_PATH_MERGE);
  if (path == AK_PATH_LEARNED)
    return run_learned(AK_OP_SORT, d_keys, d_keys, nullptr, 0, n, ki, order, d_temp, temp_bytes, st, o);
  return run_radix(AK_OP_SORT, d_keys, d_keys, nullptr, nullptr, 0, n, ki, order, d_temp, temp_bytes, st, o);
}

ak_status ak_sortperm(const void *d_keys, uint32_t *d_perm, int64_t n, ak_dtype kd, ak_order order,
                      void *d_temp, size_t temp_bytes, ak_stream_t stream, const ak_options *opt) {
  KeyInfo ki;
  ak_options o;
  if (n < 0 || !key_info(kd, &ki) || !valid_order(order) || !resolve_options(opt, &o)) return AK_ERR_INVALID_ARG;
  if (!path_supported(ki, o)) return AK_ERR_UNSUPPORTED;
  if (n == 0) return AK_OK;
  if (n > int64_t(0xFFFFFFFFll)) return AK_ERR_INDEX_OVERFLOW;
  if (!d_keys || !d_perm || !aligned(d_keys, ki.bytes) || !aligned(d_perm, 4)) return AK_ERR_INVALID_ARG;
  if (d_temp && !aligned(d_temp, 256)) return AK_ERR_INVALID_ARG;
  apply_tuning(AK_OP_SORTPERM, kd, n, 4, o);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int path = choose_path(AK_OP_SORTPERM, n, ki.bytes, 4, o);
  if (path == AK_PATH_BLOCK || path == AK_PATH_MERGE)
    return run_seg(AK_OP_SORTPERM, nullptr, nullptr, 1, n, d_keys, d_perm, 4, ki, order, d_temp, temp_bytes, st,
                   path == AK_PATH_MERGE);
  if (path == AK_PATH_LEARNED)
    return run_learned(AK_OP_SORTPERM, nullptr, d_keys, d_perm, 4, n, ki, order, d_temp, temp_bytes, st, o);
  return run_radix(AK_OP_SORTPERM, d_keys, nullptr, nullptr, d_perm, 4, n, ki, order, d_temp, temp_bytes, st, o);
}

ak_status ak_sortperm_lowmem(const void *d_keys, uint32_t *d_perm, int64_t n, ak_dtype kd, ak_order order,
                             void *d_temp, size_t temp_bytes, ak_stream_t stream, const ak_options *opt) {
  KeyInfo ki;
  ak_options o;
  if (n < 0 || !key_info(kd, &ki) || !valid_order(order) || !resolve_options(opt, &o)) return AK_ERR_INVALID_ARG;
  if (n == 0) return AK_OK;
  if (n > int64_t(0xFFFFFFFFll)) return AK_ERR_INDEX_OVERFLOW;
  if (!d_keys || !d_perm || !aligned(d_keys, ki.bytes) || !aligned(d_perm, 4)) return AK_ERR_INVALID_ARG;
  if (d_temp && !aligned(d_temp, 256)) return AK_ERR_INVALID_ARG;
  return run_radix(AK_OP_SORTPERM_LOWMEM, d_keys, nullptr, nullptr, d_perm, 4, n, ki, order, d_temp, temp_bytes,
                   reinterpret_cast<cudaStream_t>(stream), o);
}

ak_status ak_sort_pairs(void *d_keys, void *d_vals, int val_bytes, int64_t n, ak_dtype kd, ak_order order,
                        void *d_temp, size_t temp_bytes, ak_stream_t stream, const ak_options *opt) {
  KeyInfo ki;
  ak_options o;
  if (n < 0 || !key_info(kd, &ki) || !valid_order(order) || !resolve_options(opt, &o)) return AK_ERR_INVALID_ARG;
  if (val_bytes != 1 && val_bytes != 2 && val_bytes != 4 && val_bytes != 8) return AK_ERR_INVALID_ARG;
  if (!path_supported(ki, o)) return AK_ERR_UNSUPPORTED;
  if (n == 0) return AK_OK;
  if (!d_keys || !d_vals || !aligned(d_keys, ki.bytes) || !aligned(d_vals, val_bytes)) return AK_ERR_INVALID_ARG;
  if (d_temp && !aligned(d_temp, 256)) return AK_ERR_INVALID_ARG;
  apply_tuning(AK_OP_SORT_PAIRS, kd, n, val_bytes, o);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int path = choose_path(AK_OP_SORT_PAIRS, n, ki.bytes, val_bytes, o);
  if (path == AK_PATH_BLOCK || path == AK_PATH_MERGE)
    return run_seg(AK_OP_SORT_PAIRS, d_keys, nullptr, 1, n, nullptr, d_vals, val_bytes, ki, order, d_temp,
                   temp_bytes, st, path == AK_PATH_MERGE);
  if (path == AK_PATH_LEARNED)
    return run_learned(AK_OP_SORT_PAIRS, d_keys, d_keys, d_vals, val_bytes, n, ki, order, d_temp, temp_bytes, st,
                       o);
  return run_radix(AK_OP_SORT_PAIRS, d_keys, d_keys, d_vals, d_vals, val_bytes, n, ki, order, d_temp, temp_bytes,
                   st, o);
}

ak_status ak_sort_segmented(void *d_keys, const int64_t *d_offsets, int64_t nseg, int64_t n, ak_dtype kd,
                            ak_order order, void *d_temp, size_t temp_bytes, ak_stream_t stream,
                            const ak_options *opt) {
  KeyInfo ki;
  ak_options o;  // the segmented sort has no options of its own; malformed ones are still refused
  if (n < 0 || nseg < 0 || !key_info(kd, &ki) || !valid_order(order) || !resolve_options(opt, &o))
    return AK_ERR_INVALID_ARG;
  if (ki.bytes == 16) return AK_ERR_UNSUPPORTED;
  if (n == 0 || nseg == 0) return AK_OK;
  if (n > int64_t(0xFFFFFFFFll) || nseg > int64_t(0xFFFFFFFFll)) return AK_ERR_UNSUPPORTED;
  if (!d_keys || !d_offsets || !aligned(d_keys, ki.bytes) || !aligned(d_offsets, 8)) return AK_ERR_INVALID_ARG;
  if (d_temp && !aligned(d_temp, 256)) return AK_ERR_INVALID_ARG;
  int caps = o.split_caps;
  if (caps == 0 && !tune_lookup_segmented(kd, n, nseg, &caps)) caps = SPLIT_MIN_CAPS;
  const int64_t cap = seg_cap(ki.bytes, 0);
  return run_seg(AK_OP_SORT_SEGMENTED, d_keys, d_offsets, nseg, n, nullptr, nullptr, 0, ki, order, d_temp,
                 temp_bytes, reinterpret_cast<cudaStream_t>(stream), 0, caps < 0 ? -1 : int64_t(caps) * cap);
}

ak_status ak_status_check(const void *d_temp, ak_stream_t stream) {
  if (!d_temp) return AK_ERR_INVALID_ARG;
  uint32_t s = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&s, d_temp, sizeof(s), cudaMemcpyDeviceToHost, st) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return AK_ERR_CUDA;
  return static_cast<ak_status>(s);
}

ak_status ak_last_info(const void *d_temp, ak_stream_t stream, ak_info *info) {
  if (!d_temp || !info) return AK_ERR_INVALID_ARG;
  DevHeader h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&h, d_temp, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return AK_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return AK_ERR_CUDA;
  *info = h.info;
  info->status = int32_t(h.status);
  return AK_OK;
}

}  // extern "C"
