/*
 * ak_sort.h -- C ABI of a single-device GPU sort for NVIDIA GB300 (sm_103a).
 *
 * The library sorts large arrays of primitive numeric keys on one GPU: the
 * rank-local sorting step that every accelerator runs inside the sample sort of
 * the paper's distributed benchmark (Sec. IV-A, "MPISort Algorithm"), with the
 * operations of the paper's sorting building blocks (Sec. II-B: merge_sort,
 * merge_sort_by_key, sortperm) and Julia Base ordering (Sec. II).
 *
 * Ordering.  Keys are ordered by Julia `isless`: integers by value; floats by
 * value except that -0.0 sorts before +0.0 and every NaN sorts after +Inf, all
 * NaNs being equivalent.  AK_DESCENDING is Julia's rev=true: the order relation is
 * reversed (NaNs first) and equivalent keys still keep their input order.  Every
 * operation is stable, and raw key bits are moved, so NaN payloads and signs
 * survive in input order.
 *
 * Memory.  The caller owns every buffer.  The library never allocates or frees
 * device memory: each call takes a caller workspace `d_temp` whose size is given
 * ahead of time by ak_sort_temp_bytes (the "exposed temporaries" of Sec. II-B).
 * All device pointers must be device-accessible (cudaMalloc or a torch CUDA
 * tensor); `d_temp` must be 256-byte aligned.  Key, value and permutation
 * pointers must be aligned to their element size; 16-byte alignment enables the
 * bulk-copy tile loads (other alignments take plain loads).
 *
 * Asynchrony and errors.  Every call only enqueues work on `stream` (NULL = the
 * legacy default stream) and returns.  Argument errors are returned directly and
 * nothing is enqueued.  Faults found on the device (a bounded wait that expired)
 * are written to a status word inside `d_temp` and read by ak_status_check.  No
 * call synchronises the stream except ak_status_check and ak_last_info, and no
 * call allocates, so the sort calls can be captured into a CUDA graph.
 * Concurrent calls must use distinct `d_temp` buffers.
 */
#ifndef AK_SORT_H
#define AK_SORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ak_stream_t; /* same handle as cudaStream_t */

/* Key element types: the paper's FFI list (Sec. IV: int16, int32, int64,
 * float, double) with unsigned variants, and the 16-bit floats IEEE binary16
 * (AK_F16) and bfloat16 (AK_BF16, the upper half of a binary32), ordered like
 * the other floats (-0.0 before +0.0, every NaN after +Inf and tied), and the
 * 128-bit integers (AK_I128, AK_U128: two's complement, little-endian, 16-byte
 * aligned; the same layout as __int128 / unsigned __int128 on both host
 * architectures).  ak_accumulate takes neither the 16-bit floats nor the
 * 128-bit integers; 128-bit keys go through the radix path only: sort,
 * sortperm, sortperm_lowmem, sort_pairs and the binary search (segmented sort,
 * the learned, block and merge paths: AK_ERR_UNSUPPORTED). */
typedef enum ak_dtype {
    AK_U16 = 0, AK_I16 = 1, AK_U32 = 2, AK_I32 = 3,
    AK_U64 = 4, AK_I64 = 5, AK_F32 = 6, AK_F64 = 7,
    AK_F16 = 8, AK_BF16 = 9, AK_I128 = 10, AK_U128 = 11
} ak_dtype;

typedef enum ak_order { AK_ASCENDING = 0, AK_DESCENDING = 1 } ak_order;

typedef enum ak_status {
    AK_OK = 0,
    AK_ERR_INVALID_ARG = 1,         /* NULL pointer with n > 0, bad enum, bad size */
    AK_ERR_UNSUPPORTED = 2,         /* valid request this build does not serve */
    AK_ERR_WORKSPACE_TOO_SMALL = 3, /* d_temp NULL or temp_bytes too small */
    AK_ERR_CUDA = 4,                /* a CUDA runtime call or launch failed */
    AK_ERR_TIMEOUT = 5,             /* a device-side wait exceeded its bound */
    AK_ERR_INDEX_OVERFLOW = 6       /* sortperm with n >= 2^32 (UInt32 indices) */
} ak_status;

typedef enum ak_op {
    AK_OP_SORT = 0, AK_OP_SORTPERM = 1, AK_OP_SORT_PAIRS = 2, AK_OP_SORT_SEGMENTED = 3,
    AK_OP_SORTPERM_LOWMEM = 4
} ak_op;

typedef enum ak_path {
    AK_PATH_AUTO = 0,     /* library choice (autotune cache, then size rules) */
    AK_PATH_RADIX = 1,    /* onesweep LSD radix: histogram + one kernel per digit */
    AK_PATH_LEARNED = 2,  /* learned-CDF bucketing + per-bucket shared-memory sort */
    AK_PATH_BLOCK = 3,    /* one-launch shared-memory sort (small n only) */
    AK_PATH_MERGE = 4     /* tiles of the shared-memory capacity sorted in one launch, then
                             stable merge-path rounds (mid-size n) */
} ak_path;

/* Optional tuning knobs.  Pass NULL for defaults; zero fields mean "default".
 * A field outside its documented range (unknown path, tile configuration or
 * debug flag, bucket_bits not 0 or 8..16, train_steps below -1, digit_bits not 0
 * or 8, split_caps outside -1..1024, a nonzero reserved word) makes the call
 * return AK_ERR_INVALID_ARG with nothing
 * enqueued; the options are checked before the n = 0 early return, so an
 * empty call with malformed options is refused too. */
typedef struct ak_options {
    int32_t path;          /* ak_path */
    int32_t tile_config;   /* digit-pass variant, 0 = default (1), else 1..AK_TILE_CONFIGS:
                              1 persistent 512-thread CTAs, 40 KB tiles; 2 persistent
                              384-thread CTAs, 24 KB tiles; 3 one 512-thread CTA per
                              32 KB tile with an L2 prefetch one wave ahead; 4 persistent
                              512-thread CTAs whose last warp does the look-back while
                              the others rank the next tile (three tile buffers); 5 the
                              reduce-then-scan form of 1 (three-kernel scheme instead of
                              onesweep): per pass an upsweep kernel counts the digits of
                              each chunk of consecutive tiles, then one CTA per chunk
                              sorts its tiles in order from running digit offsets, with no
                              look-back (one more read of the keys per pass; above 2^30
                              keys it runs as 1) */
    int32_t bucket_bits;   /* learned path: log2 of the bucket count, 8..16 (NaN keys share
                              the last bucket); 0 = auto, about half the shared-memory
                              finish capacity (ak_segment_capacity) per bucket */
    uint32_t seed;         /* learned path: seed of the sample index stream */
    uint64_t timeout_ns;   /* bound on every device-side wait, 0 = 1 s */
    int32_t train_steps;   /* learned path: Adam steps of the residual MLP, 0 = default (16),
                              -1 = no MLP (piecewise-linear CDF only) */
    int32_t debug_flags;   /* test hooks, 0 in normal use (AK_DEBUG_*) */
    void **pass_events;    /* optional: 2*AK_MAX_PASSES cudaEvent_t created by the caller;
                              the radix path records [2p] before and [2p+1] after the
                              launch of digit pass p on the call's stream (profiling) */
    int32_t digit_bits;    /* radix digit width: 0 = default = 8, the only width built
                              (an 11-bit digit pass is not), so any other value is refused */
    int32_t split_caps;    /* ak_sort_segmented: segments longer than split_caps times the
                              shared-memory capacity (ak_segment_capacity) are cut into
                              buckets by all CTAs together before the per-CTA sort; shorter
                              ones above the capacity are sorted by one CTA through global
                              memory.  0 = autotuned choice, else 8; -1 = never split;
                              else 1..1024 */
    int32_t reserved[2];   /* must be zero */
} ak_options;

#define AK_MAX_PASSES 16

/* Test hook: no CTA owns the first tile of any radix pass, so every
 * look-back that reaches it waits until
 * timeout_ns and the call ends with AK_ERR_TIMEOUT (the output is then
 * unspecified).  Exercises the bounded-wait error path.  Tile configuration 5
 * has no look-back and ignores it. */
#define AK_DEBUG_SKIP_FIRST_TILE 1
/* Tuning hook: no L2 prefetch one wave ahead in tile configuration 3 (the
 * persistent configurations prefetch each claimed tile, unaffected). */
#define AK_DEBUG_NO_PREFETCH 2
/* Tuning hook: ak_sortperm of 8-byte keys moves key and index through every
 * digit pass, instead of packing the upper half of the key and the index into
 * one 8-byte word for the passes of the upper key half (the default for tile
 * configuration 1 up to 2^30 keys).  The permutation is the same. */
#define AK_DEBUG_NO_PACK 4

#define AK_TILE_CONFIGS 5

/* Diagnostics written by the device for the most recent call on a d_temp. */
typedef struct ak_info {
    int32_t status;          /* ak_status of the device side */
    int32_t path;            /* ak_path actually executed (learned may fall back to radix) */
    int32_t radix_passes;    /* digit passes that moved data (trivial passes skipped) */
    int32_t buckets;         /* learned: bucket count used */
    int64_t overfull_keys;   /* learned: keys in buckets above 16x the shared-memory capacity */
    int64_t max_bucket;      /* learned: largest bucket */
    float loss_before;       /* learned: training loss of the piecewise-linear CDF alone */
    float loss_after;        /* learned: training loss after the MLP residual is trained */
    int64_t sample_size;     /* learned: sample keys drawn */
    int64_t coordinate;      /* learned: model input, 0 radix key, 1 value of a float key */
    int32_t mlp_used;        /* learned: 1 when the bucket table holds the trained MLP residual,
                                0 when the piecewise-linear CDF alone gave the sorted sample a
                                smaller (or equal) largest bucket, or nothing was trained */
    int32_t reserved0;
    int64_t sample_max_pl;   /* learned: most sample keys in one bucket, piecewise-linear table */
    int64_t sample_max_mlp;  /* learned: the same with the MLP residual (0: not trained) */
} ak_info;

/*
 * Workspace bytes for one call.
 *   op        ak_op
 *   n         number of keys (>= 0)
 *   kd        key dtype
 *   val_bytes AK_OP_SORT_PAIRS: bytes per value (1, 2, 4 or 8); ignored otherwise
 *   nseg      AK_OP_SORT_SEGMENTED: number of segments; ignored otherwise
 *   opt       options (NULL = defaults); the path changes the size
 *   bytes     out: required size of d_temp
 * Returns AK_ERR_INVALID_ARG for a negative n/nseg, a bad enum or a NULL `bytes`.
 */
ak_status ak_sort_temp_bytes(int op, int64_t n, ak_dtype kd, int val_bytes, int64_t nseg,
                             const ak_options *opt, size_t *bytes);

/*
 * In-place stable sort of d_keys[0..n) (Sec. II-B "merge_sort"; the local sort of
 * Sec. IV-A).  n = 0 is a no-op.
 */
ak_status ak_sort(void *d_keys, int64_t n, ak_dtype kd, ak_order order,
                  void *d_temp, size_t temp_bytes, ak_stream_t stream, const ak_options *opt);

/*
 * Stable sorting permutation (Sec. II-B "sortperm"): d_perm[i] is the 0-based
 * index of the key that belongs at position i.  d_keys is read only.  Indices are
 * UInt32, so n >= 2^32 returns AK_ERR_INDEX_OVERFLOW.  d_perm must not overlap
 * d_keys or d_temp.  For 8-byte keys (up to 2^30, default tile configuration)
 * the radix passes over the upper 32 key bits move one 8-byte word per key,
 * the upper half of the order-preserving key over the index, instead of the key
 * and the index; AUTO takes that radix path for them.
 */
ak_status ak_sortperm(const void *d_keys, uint32_t *d_perm, int64_t n, ak_dtype kd, ak_order order,
                      void *d_temp, size_t temp_bytes, ak_stream_t stream, const ak_options *opt);

/*
 * ak_sortperm with less temporary memory (Sec. II-B "sortperm_lowmem"): the
 * same permutation, bit for bit, from a workspace that holds no copy of the
 * keys (ak_sort_temp_bytes with AK_OP_SORTPERM_LOWMEM: about n * 4 bytes plus
 * per-tile counters, where ak_sortperm needs 2 n * key bytes more).  Every
 * digit pass moves only the indices and reads each key through its index from
 * d_keys, so the passes after the first gather keys from anywhere in d_keys
 * (slower than ak_sortperm).  Always the radix path; tile_config 4 and 5 run as 1.
 * Arguments, errors and limits as ak_sortperm.
 */
ak_status ak_sortperm_lowmem(const void *d_keys, uint32_t *d_perm, int64_t n, ak_dtype kd, ak_order order,
                             void *d_temp, size_t temp_bytes, ak_stream_t stream, const ak_options *opt);

/*
 * In-place stable key-value sort (Sec. II-B "merge_sort_by_key"): keys and the
 * values d_vals[0..n) (val_bytes = 1, 2, 4 or 8 each) are permuted together.
 */
ak_status ak_sort_pairs(void *d_keys, void *d_vals, int val_bytes, int64_t n, ak_dtype kd,
                        ak_order order, void *d_temp, size_t temp_bytes, ak_stream_t stream,
                        const ak_options *opt);

/*
 * Segmented in-place stable sort: every CSR segment d_keys[off[s], off[s+1]),
 * s < nseg, is sorted on its own, all in one batch of launches.  d_offsets is a
 * device array of nseg+1 int64 values, non-decreasing, off[0] = 0 and
 * off[nseg] = n.  The offsets are read on the device only; offsets that break
 * these rules leave the keys of the affected segments unspecified (never an
 * out-of-bounds access: every offset is clamped to [0, n]).  n and nseg above
 * 2^32 - 1 return AK_ERR_UNSUPPORTED.
 */
ak_status ak_sort_segmented(void *d_keys, const int64_t *d_offsets, int64_t nseg, int64_t n,
                            ak_dtype kd, ak_order order, void *d_temp, size_t temp_bytes,
                            ak_stream_t stream, const ak_options *opt);

/*
 * ak_sort without a caller workspace, for callers that cannot allocate device
 * memory: code running inside a CUDA stream-capture region (cudaMalloc is not
 * allowed there), latency-critical loops where cudaMalloc's implicit device
 * synchronisation is unacceptable, and hosts whose device memory is owned by a
 * framework pool that forbids foreign allocations.  There is no counterpart in
 * the paper; it exists for these callers only.
 *
 * The workspace is a static device array of AK_STATIC_SCRATCH_BYTES inside this
 * library; every GPU that loads the library holds it until the process exits.
 * Requests whose ak_sort workspace (ak_sort_temp_bytes with AK_OP_SORT) exceeds
 * it return AK_ERR_WORKSPACE_TOO_SMALL with nothing enqueued.  The call allocates
 * nothing.  Its first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it, so make that first call before any stream
 * capture.  All calls share the one array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.  Results,
 * ordering and stability are those of ak_sort; device-side timeouts are recorded
 * only in the shared array and are not returned (a caller that needs them uses
 * ak_sort with its own workspace and ak_status_check).  The cached address is
 * that of the device's current context: a device reset (cudaDeviceReset, or
 * the primary context destroyed and re-created) is not supported for this entry
 * point within the same process.
 */
#define AK_STATIC_SCRATCH_BYTES (32u << 20)
ak_status ak_sort_static_scratch(void *d_keys, int64_t n, ak_dtype kd, ak_order order, ak_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Binary search (Sec. II-B, searchsortedfirst / searchsortedlast).          */

/*
 * For each of m query keys d_x[i], its place among the n keys d_v, which must
 * already be in `order`'s sequence (as ak_sort leaves them with that order).
 * "Comes before" is the sort's order: Julia isless, or its reverse for
 * AK_DESCENDING (all NaNs equivalent, -0.0 before +0.0).  Results are 0-based:
 *   ak_searchsortedfirst: d_out[i] = index of the first d_v element that does
 *     not come before d_x[i], n if none (Julia's searchsortedfirst minus one):
 *     the insertion index in front of every key equivalent to d_x[i];
 *   ak_searchsortedlast:  d_out[i] = index of the last d_v element that d_x[i]
 *     does not come before, -1 if none (Julia's searchsortedlast minus one);
 *     plus one it is the insertion index behind every equivalent key.
 * d_v (n keys) and d_x (m keys) are device arrays of dtype kd aligned to the
 * key size; they may be the same array.  d_out is m int64 on the device,
 * 8-byte aligned, overlapping neither.  Both functions only enqueue one kernel
 * on `stream`: no workspace, no allocation, no synchronisation (graph
 * capturable).  If d_v is not in order the results are unspecified but stay in
 * [0, n] (first) or [-1, n - 1] (last), and nothing outside d_v[0, n) is read.
 * n = 0 is valid (every result 0, or -1); m = 0 enqueues nothing.
 * Returns AK_ERR_INVALID_ARG for a negative n or m, a bad dtype or order, or a
 * NULL or misaligned pointer that would be read or written; AK_ERR_CUDA if the
 * launch fails.
 */
ak_status ak_searchsortedfirst(const void *d_v, int64_t n, const void *d_x, int64_t m, ak_dtype kd,
                               ak_order order, int64_t *d_out, ak_stream_t stream);
ak_status ak_searchsortedlast(const void *d_v, int64_t n, const void *d_x, int64_t m, ak_dtype kd,
                              ak_order order, int64_t *d_out, ak_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Accumulate (Sec. II-B: prefix scan, inclusive and exclusive, with          */
/* decoupled look-back).                                                      */

typedef enum ak_scan_op { AK_SCAN_ADD = 0, AK_SCAN_MAX = 1, AK_SCAN_MIN = 2 } ak_scan_op;

/*
 * Prefix scan of the n keys d_x into d_out, both of dtype kd:
 *   inclusive = 1: d_out[i] = init (+) d_x[0] (+) ... (+) d_x[i]
 *   inclusive = 0: d_out[i] = init (+) d_x[0] (+) ... (+) d_x[i-1], d_out[0] = init
 * where (+) is
 *   AK_SCAN_ADD  integer + wrapping in the key's width; IEEE float + in the key's
 *                precision, in an order of its own (results differ from a left
 *                to right sum by rounding only: the bound is that of a sum of
 *                depth at most m + 2 ceil(n / (32768 m)) + 84, m = 64 / key
 *                bytes, 16 for 16-bit keys);
 *   AK_SCAN_MAX  Julia max: a NaN operand gives NaN, +0.0 is above -0.0;
 *   AK_SCAN_MIN  Julia min: a NaN operand gives NaN, -0.0 is below +0.0.
 * Integer results and max/min are exact.
 * h_init is a HOST pointer to one key of dtype kd, or NULL for the operator's
 * identity (0 or -0.0 for +; the lowest value or -Inf for max; the highest
 * or +Inf for min).  d_out may be d_x (in place) but must not otherwise
 * overlap it.  Pointers are aligned to the key size (16-byte alignment of both
 * enables vector loads).  d_temp: a 256-byte aligned workspace of
 * ak_accumulate_temp_bytes bytes, whose first bytes hold the status word that
 * ak_status_check reads (always AK_OK: no kernel of the scan waits on another
 * CTA); opt may be NULL, and its timeout_ns and debug_flags have no effect here.
 * Enqueues one memset and three kernels on `stream` (range totals, their
 * prefixes, the ranges' scans); allocates nothing.
 * Returns AK_ERR_INVALID_ARG for a negative n, a bad dtype, op or inclusive
 * flag, malformed options, or a NULL or misaligned pointer with n > 0;
 * AK_ERR_WORKSPACE_TOO_SMALL; AK_ERR_CUDA if a launch fails.  n = 0 is a no-op.
 */
ak_status ak_accumulate(const void *d_x, void *d_out, int64_t n, ak_dtype kd, ak_scan_op op, int inclusive,
                        const void *h_init, void *d_temp, size_t temp_bytes, ak_stream_t stream,
                        const ak_options *opt);
/* Workspace bytes ak_accumulate needs for n keys of dtype kd (host only). */
ak_status ak_accumulate_temp_bytes(int64_t n, ak_dtype kd, size_t *bytes);

/*
 * Synchronises `stream` and returns the device-side status of the last call that
 * used d_temp (AK_OK, or e.g. AK_ERR_TIMEOUT).  AK_ERR_CUDA if the copy fails.
 */
ak_status ak_status_check(const void *d_temp, ak_stream_t stream);

/* Synchronises `stream` and copies the diagnostics of the last call on d_temp. */
ak_status ak_last_info(const void *d_temp, ak_stream_t stream, ak_info *info);

/* Static English description of a status code. */
const char *ak_status_string(ak_status s);

/* ------------------------------------------------------------------------- */
/* Learned-CDF model kernels, exposed for checking against a CPU restatement. */
/* The sample-sort splitter step (Sec. IV-A) draws the sample these act on.  */

#define AK_LEARNED_KNOTS 64
#define AK_LEARNED_PARAMS 321

/*
 * Knots of the piecewise-linear CDF: d_knots[j] = d_xs[round(j (m-1) / 63)],
 * j < 64, for an ascending float32 sample d_xs[0..m) of x-hat values in [0, 1]:
 * the sample order statistics that the sample sort's splitter step picks
 * (Sec. IV-A), through which PL interpolates (xi_j, j/63).  m >= 1.
 */
ak_status ak_learned_knots(const float *d_xs, int64_t m, float *d_knots, ak_stream_t stream);

/*
 * Loss and gradient of the residual MLP (1 -> 16 -> 16 -> 1, ReLU, output scaled
 * by 1/1024) for the model F(x) = PL(x) + r(x): d_loss[0] = mean_i (F(x_i) - y_i)^2 and d_grad = dLoss/dparams,
 * computed by the same forward/backward kernels the learned path trains with.
 *   d_x, d_y   m float32 inputs and targets
 *   d_c        64 float32 PL knots xi_j (non-decreasing), PL(xi_j) = j/63
 *   d_params   321 float32: W1[16], b1[16], W2[16][16] (row j feeds hidden unit j),
 *              b2[16], w3[16], b3
 *   d_grad     321 float32 out; d_loss 1 float32 out
 *   d_temp     workspace of at least ak_learned_grad_temp_bytes(m) bytes
 * The reduction order is fixed, so results are deterministic.
 */
ak_status ak_learned_loss_grad(const float *d_x, const float *d_y, int64_t m, const float *d_c,
                               const float *d_params, float *d_grad, float *d_loss,
                               void *d_temp, size_t temp_bytes, ak_stream_t stream);
size_t ak_learned_grad_temp_bytes(int64_t m);

/* ------------------------------------------------------------------------- */
/* Autotuner: times the onesweep tile configurations and the learned and block
 * paths on the caller's buffers and caches the fastest per (op, dtype,
 * ceil(log2 n), value bytes).  AK_PATH_AUTO calls with tile_config 0 (and
 * ak_sort_temp_bytes for them) take the cached choice; the environment variable
 * AK_TUNE_CACHE names a cache file loaded on first use. */

/*
 * Tunes one call shape (op = AK_OP_SORT, AK_OP_SORTPERM or AK_OP_SORT_PAIRS):
 * times the radix path in each tile configuration, the learned path at its own
 * bucket count and at half and twice as many buckets, and the block path when n
 * fits one CTA (else the merge path up to 2^26 keys), and caches the fastest
 * (path, tile configuration, bucket bits).
 * d_keys (and d_vals for pairs, d_perm for sortperm) are the call's buffers: they
 * are restored from a copy before every timed call and hold the original inputs
 * again on return.  d_temp must hold ak_autotune_temp_bytes bytes (the largest
 * candidate's workspace, rounded up to 256 bytes, plus n * (key bytes + value
 * bytes) for the copy).  Synchronises `stream`.  `best` (optional) receives the
 * chosen options.
 */
ak_status ak_autotune(int op, int64_t n, ak_dtype kd, int val_bytes, ak_order order,
                      void *d_keys, void *d_vals, uint32_t *d_perm, void *d_temp,
                      size_t temp_bytes, ak_stream_t stream, ak_options *best);
/* Workspace ak_autotune needs for this call shape (host only). */
ak_status ak_autotune_temp_bytes(int op, int64_t n, ak_dtype kd, int val_bytes, size_t *bytes);

/*
 * Tunes ak_sort_segmented for the caller's batch: times the split threshold
 * (split_caps 1, 2, 4, 8, 16 and never) on d_keys / d_offsets (restored from a
 * copy before every timed call; the keys hold their input again on return) and
 * caches the fastest under (dtype, ceil(log2 n), ceil(log2 nseg)); segmented
 * calls with split_caps 0 take it.  d_temp: ak_autotune_segmented_temp_bytes
 * bytes.  Synchronises `stream`.  `best` (optional) receives the choice.
 */
ak_status ak_autotune_segmented(void *d_keys, const int64_t *d_offsets, int64_t nseg, int64_t n, ak_dtype kd,
                                ak_order order, void *d_temp, size_t temp_bytes, ak_stream_t stream,
                                ak_options *best);
ak_status ak_autotune_segmented_temp_bytes(int64_t n, int64_t nseg, ak_dtype kd, size_t *bytes);
/* The cache as JSON lines {"op", "dtype", "log2n", "val_bytes", "path",
 * "tile_config", "ms", "bucket_bits", "split_caps"} (bucket_bits and split_caps
 * optional, 0 = automatic; segmented entries have op 3 and ceil(log2 nseg) in
 * val_bytes): save, load (merging; malformed lines are skipped), clear. */
ak_status ak_autotune_save(const char *path);
ak_status ak_autotune_load(const char *path);
void ak_autotune_clear(void);

/* Library version string. */
const char *ak_version(void);

/* Keys of one segment that the segmented sort (and AK_PATH_BLOCK) sorts in
 * shared memory, for keys of key_bytes (2, 4, 8) and values of val_bytes (0, 1,
 * 2, 4, 8; ak_sortperm carries 4-byte indices).  Longer segments first take an
 * MSD split through global memory (the workspace copy of the segment).  Returns
 * 0 for unsupported widths. */
int64_t ak_segment_capacity(int key_bytes, int val_bytes);

#ifdef __cplusplus
}
#endif

#endif /* AK_SORT_H */
