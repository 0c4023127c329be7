/*
 * ak_oracle.c -- CPU oracle for the single-device sort.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
 * baseline use this file.  It shares no code, header, table or helper with the
 * CUDA library and must never be reached from the library's product path.
 *
 * What it computes (the definition, written out):
 *   For keys k[0..n) the result is the unique STABLE permutation p such that for
 *   every i < j either lt(k[p[i]], k[p[j]]) holds, or neither lt(k[p[i]], k[p[j]])
 *   nor lt(k[p[j]], k[p[i]]) holds and p[i] < p[j].
 *   lt is Julia's isless for ascending order and lt(a,b) = isless(b,a) for
 *   descending order (Julia's rev=true, which keeps equal keys in input order).
 *   sort        -> k o p            (the local sort of Sec. IV-A)
 *   sortperm    -> p                (Sec. II-B, "sortperm")
 *   sort_pairs  -> (k o p, v o p)   (Sec. II-B, "merge_sort_by_key")
 *   segmented   -> the same definition applied to every CSR segment alone.
 *
 * Julia isless on integers is <.  On IEEE floats: every NaN compares after every
 * non-NaN and all NaNs are equivalent; -0.0 comes before +0.0; otherwise <.
 * Key types: 16/32/64/128-bit integers, float32, float64, and the 16-bit floats
 * (IEEE binary16 and bfloat16, compared through their exact float32 values).
 *
 *   searchsortedfirst / searchsortedlast (Sec. II-B, binary search) -> for a v
 *   already in the order's sequence, the 0-based index of the first element of
 *   v that does not come before x, and of the last element that x does not come
 *   before (Julia's 1-based results minus one).
 *   accumulate (Sec. II-B, prefix scan) -> inclusive or exclusive running
 *   +, max or min from a start value, left to right (details at the function).
 *
 * How: a textbook top-down merge sort on an index array.  The merge takes the
 * right element only when it is strictly less than the left one, so ties keep
 * input order.  A threaded variant sorts equal chunks in parallel and merges
 * them pairwise with the same merge.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OD_U16 = 0, OD_I16, OD_U32, OD_I32, OD_U64, OD_I64, OD_F32, OD_F64, OD_F16, OD_BF16,
       OD_I128, OD_U128, OD_COUNT };

typedef struct {
    const void *keys;
    int dtype;
    int descending;
} oracle_ctx;

/* Julia isless for floats of either width. */
static int isless_double(double a, double b) {
    if (isnan(a)) return 0;          /* NaN is never less than anything */
    if (isnan(b)) return 1;          /* every non-NaN is less than NaN */
    if (a < b) return 1;
    if (a == b) return signbit(a) && !signbit(b);   /* -0.0 before +0.0 */
    return 0;
}

static int isless_float(float a, float b) {
    if (isnan(a)) return 0;
    if (isnan(b)) return 1;
    if (a < b) return 1;
    if (a == b) return signbit(a) && !signbit(b);
    return 0;
}

/* IEEE 754 binary16 bits -> the same value as a float (exact): sign, 5-bit
 * exponent (bias 15), 10-bit fraction; exponent 0 is zero or subnormal
 * (fraction x 2^-24), exponent 31 is Inf (fraction 0) or NaN. */
static float half_to_float(uint16_t h) {
    const int e = (h >> 10) & 0x1F, m = h & 0x3FF;
    float v;
    if (e == 0) v = ldexpf((float)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexpf((float)(m | 0x400), e - 25);   /* (1024 + m) x 2^(e - 25) */
    return (h >> 15) ? -v : v;
}

/* bfloat16 bits are the top half of a float32's bits (exact). */
static float bf16_to_float(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

/* 128-bit integers, 16 bytes each (low 8 bytes first), read with memcpy so
 * that any alignment of the caller's array is fine. */
static __int128 load_i128(const void *p, int64_t i) {
    __int128 v;
    memcpy(&v, (const unsigned char *)p + (size_t)i * 16, 16);
    return v;
}
static unsigned __int128 load_u128(const void *p, int64_t i) {
    unsigned __int128 v;
    memcpy(&v, (const unsigned char *)p + (size_t)i * 16, 16);
    return v;
}

/* isless(a[i], b[j]) for keys of one dtype held in two arrays */
static int isless_at(int dtype, const void *a, int64_t i, const void *b, int64_t j) {
    switch (dtype) {
    case OD_U16: return ((const uint16_t *)a)[i] < ((const uint16_t *)b)[j];
    case OD_I16: return ((const int16_t *)a)[i] < ((const int16_t *)b)[j];
    case OD_U32: return ((const uint32_t *)a)[i] < ((const uint32_t *)b)[j];
    case OD_I32: return ((const int32_t *)a)[i] < ((const int32_t *)b)[j];
    case OD_U64: return ((const uint64_t *)a)[i] < ((const uint64_t *)b)[j];
    case OD_I64: return ((const int64_t *)a)[i] < ((const int64_t *)b)[j];
    case OD_F32: return isless_float(((const float *)a)[i], ((const float *)b)[j]);
    case OD_F64: return isless_double(((const double *)a)[i], ((const double *)b)[j]);
    case OD_F16: return isless_float(half_to_float(((const uint16_t *)a)[i]), half_to_float(((const uint16_t *)b)[j]));
    case OD_BF16: return isless_float(bf16_to_float(((const uint16_t *)a)[i]), bf16_to_float(((const uint16_t *)b)[j]));
    case OD_I128: return load_i128(a, i) < load_i128(b, j);
    case OD_U128: return load_u128(a, i) < load_u128(b, j);
    }
    return 0;
}

/* isless(key[i], key[j]) */
static int key_isless(const oracle_ctx *c, int64_t i, int64_t j) {
    return isless_at(c->dtype, c->keys, i, c->keys, j);
}

/* the order's strict "comes before": isless, or isless with operands swapped */
static int lt(const oracle_ctx *c, int64_t i, int64_t j) {
    return c->descending ? key_isless(c, j, i) : key_isless(c, i, j);
}

/* Merge idx[lo,mid) and idx[mid,hi) (each already in order) through tmp. */
static void merge_runs(const oracle_ctx *c, int64_t *idx, int64_t *tmp,
                       int64_t lo, int64_t mid, int64_t hi) {
    int64_t a = lo, b = mid, o = lo;
    while (a < mid && b < hi) {
        if (lt(c, idx[b], idx[a])) tmp[o++] = idx[b++];   /* right strictly first */
        else tmp[o++] = idx[a++];                         /* ties: left first */
    }
    while (a < mid) tmp[o++] = idx[a++];
    while (b < hi) tmp[o++] = idx[b++];
    memcpy(idx + lo, tmp + lo, (size_t)(hi - lo) * sizeof(int64_t));
}

static void merge_sort(const oracle_ctx *c, int64_t *idx, int64_t *tmp, int64_t lo, int64_t hi) {
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    merge_sort(c, idx, tmp, lo, mid);
    merge_sort(c, idx, tmp, mid, hi);
    merge_runs(c, idx, tmp, lo, mid, hi);
}

static int check_args(const void *keys, int64_t n, int dtype, const int64_t *perm) {
    if (n < 0 || dtype < 0 || dtype >= OD_COUNT) return -1;
    if (n > 0 && (!keys || !perm)) return -1;
    return 0;
}

/* perm[0..n) <- the stable sorting permutation of keys (0-based). */
int oracle_sortperm(const void *keys, int64_t n, int dtype, int descending, int64_t *perm) {
    if (check_args(keys, n, dtype, perm)) return -1;
    oracle_ctx c = {keys, dtype, descending};
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    if (n < 2) return 0;
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!tmp) return -2;
    merge_sort(&c, perm, tmp, 0, n);
    free(tmp);
    return 0;
}

/* ---------------------------------------------------------------- threaded -- */
typedef struct {
    const oracle_ctx *c;
    int64_t *idx, *tmp;
    int64_t lo, mid, hi;
    int merge_only;
} oracle_job;

static void *oracle_job_run(void *p) {
    oracle_job *j = (oracle_job *)p;
    if (j->merge_only) merge_runs(j->c, j->idx, j->tmp, j->lo, j->mid, j->hi);
    else merge_sort(j->c, j->idx, j->tmp, j->lo, j->hi);
    return NULL;
}

/* Same result as oracle_sortperm: `nthreads` equal chunks sorted in parallel,
 * then merged pairwise (left run first on ties), level by level. */
int oracle_sortperm_threaded(const void *keys, int64_t n, int dtype, int descending,
                             int64_t *perm, int nthreads) {
    if (check_args(keys, n, dtype, perm)) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 2 * (int64_t)nthreads || nthreads == 1)
        return oracle_sortperm(keys, n, dtype, descending, perm);
    oracle_ctx c = {keys, dtype, descending};
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!tmp) return -2;
    int64_t bounds[257];
    for (int t = 0; t <= nthreads; ++t) bounds[t] = n * t / nthreads;
    pthread_t th[256];
    oracle_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (oracle_job){&c, perm, tmp, bounds[t], 0, bounds[t + 1], 0};
        pthread_create(&th[t], NULL, oracle_job_run, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    /* runs are bounds[r]..bounds[r+1]; merge neighbours until one run remains */
    int runs = nthreads;
    int64_t rb[257];
    memcpy(rb, bounds, sizeof(int64_t) * (size_t)(nthreads + 1));
    while (runs > 1) {
        int pairs = runs / 2, nj = 0;
        for (int r = 0; r < pairs; ++r) {
            jobs[nj] = (oracle_job){&c, perm, tmp, rb[2 * r], rb[2 * r + 1], rb[2 * r + 2], 1};
            pthread_create(&th[nj], NULL, oracle_job_run, &jobs[nj]);
            ++nj;
        }
        for (int r = 0; r < nj; ++r) pthread_join(th[r], NULL);
        int64_t nb[257];
        int k = 0;
        for (int r = 0; r < pairs; ++r) nb[k++] = rb[2 * r];
        if (runs & 1) nb[k++] = rb[runs - 1];
        nb[k] = rb[runs];
        runs = k;
        memcpy(rb, nb, sizeof(int64_t) * (size_t)(runs + 1));
    }
    free(tmp);
    return 0;
}

/* Segmented: perm holds global indices; each CSR segment [off[s], off[s+1]) is
 * sorted on its own.  Offsets must be non-decreasing, off[0] = 0, off[nseg] = n. */
int oracle_sortperm_segmented(const void *keys, const int64_t *off, int64_t nseg, int64_t n,
                              int dtype, int descending, int64_t *perm) {
    if (check_args(keys, n, dtype, perm) || nseg < 0 || (nseg > 0 && !off)) return -1;
    if (nseg > 0 && (off[0] != 0 || off[nseg] != n)) return -1;
    for (int64_t s = 0; s < nseg; ++s)
        if (off[s + 1] < off[s]) return -1;
    oracle_ctx c = {keys, dtype, descending};
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    if (n < 2) return 0;
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!tmp) return -2;
    for (int64_t s = 0; s < nseg; ++s) merge_sort(&c, perm, tmp, off[s], off[s + 1]);
    free(tmp);
    return 0;
}

/* dst[i] = src[perm[i]] for elements of elem_bytes bytes (raw bits are moved). */
int oracle_gather(const void *src, const int64_t *perm, int64_t n, int elem_bytes, void *dst) {
    if (n < 0 || elem_bytes <= 0) return -1;
    const unsigned char *s = (const unsigned char *)src;
    unsigned char *d = (unsigned char *)dst;
    for (int64_t i = 0; i < n; ++i)
        memcpy(d + (size_t)i * (size_t)elem_bytes, s + (size_t)perm[i] * (size_t)elem_bytes,
               (size_t)elem_bytes);
    return 0;
}

/* isless(a[i], b[i]) for n pairs, exposed so tests can pin the comparator itself. */
int oracle_isless_pairs(const void *a, const void *b, int64_t n, int dtype, uint8_t *out) {
    if (n < 0 || dtype < 0 || dtype >= OD_COUNT) return -1;
    size_t w = (dtype <= OD_I16 || dtype == OD_F16 || dtype == OD_BF16) ? 2
             : (dtype <= OD_I32 || dtype == OD_F32) ? 4
             : (dtype == OD_I128 || dtype == OD_U128) ? 16 : 8;
    unsigned char *buf = (unsigned char *)malloc(2 * w);
    if (!buf) return -2;
    oracle_ctx c = {buf, dtype, 0};
    for (int64_t i = 0; i < n; ++i) {
        memcpy(buf, (const unsigned char *)a + (size_t)i * w, w);
        memcpy(buf + w, (const unsigned char *)b + (size_t)i * w, w);
        out[i] = (uint8_t)key_isless(&c, 0, 1);
    }
    free(buf);
    return 0;
}

/* Binary search, Sec. II-B (searchsortedfirst / searchsortedlast), over keys
 * v[0..n) that are already in the order's sequence (isless ascending, or its
 * reverse for descending).  For every query x[i]:
 *   side 0: out[i] = index of the first v element that does not come before
 *           x[i], n if there is none (Julia's searchsortedfirst minus one);
 *   side 1: out[i] = index of the last v element that x[i] does not come
 *           before, -1 if there is none (Julia's searchsortedlast minus one).
 * Textbook bisection on [lo, hi): the predicate "v[mid] comes before x" (side
 * 0) or "x does not come before v[mid]" (side 1) holds on a prefix of a sorted
 * v, and lo ends at the length of that prefix. */
int oracle_searchsorted(const void *v, int64_t n, const void *x, int64_t m, int dtype,
                        int descending, int side, int64_t *out) {
    if (n < 0 || m < 0 || dtype < 0 || dtype >= OD_COUNT || (side != 0 && side != 1)) return -1;
    if ((n > 0 && !v) || (m > 0 && (!x || !out))) return -1;
    for (int64_t i = 0; i < m; ++i) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            int in_prefix;
            if (side == 0)   /* v[mid] before x */
                in_prefix = descending ? isless_at(dtype, x, i, v, mid) : isless_at(dtype, v, mid, x, i);
            else             /* x not before v[mid] */
                in_prefix = !(descending ? isless_at(dtype, v, mid, x, i) : isless_at(dtype, x, i, v, mid));
            if (in_prefix) lo = mid + 1;
            else hi = mid;
        }
        out[i] = side == 0 ? lo : lo - 1;
    }
    return 0;
}

/* -------------------------------------------------------------- accumulate -- */
/* Prefix scan, Sec. II-B (accumulate), with a start value `init`:
 *   inclusive: out[i] = init (+) x[0] (+) ... (+) x[i]
 *   exclusive: out[i] = init (+) x[0] (+) ... (+) x[i-1]   (out[0] = init)
 * for (+) one of
 *   OA_ADD  integer +, wrapping in the key's width (Julia's integer +); float
 *           +, summed in float64 with Neumaier's compensation (Neumaier 1974,
 *           "Rundungsfehleranalyse einiger Verfahren zur Summation endlicher
 *           Summen") and each output rounded once to the key's type -- the
 *           mathematical prefix sum to well within one rounding.  While the
 *           compensation is zero the output is the running float64 sum itself
 *           (so sums of -0.0 stay -0.0); once that running sum is not finite
 *           (a NaN or an infinity in the prefix, or overflow) the output is
 *           that running sum;
 *   OA_MAX  Julia max: NaN if either operand is NaN, +0.0 above -0.0;
 *   OA_MIN  Julia min: NaN if either operand is NaN, -0.0 below +0.0.
 * Written strictly left to right, one element at a time. */
enum { OA_ADD = 0, OA_MAX = 1, OA_MIN = 2 };

static double julia_max(double a, double b) {
    if (isnan(a)) return a;
    if (isnan(b)) return b;
    if (a == b) return signbit(a) ? b : a;   /* max(-0.0, 0.0) = 0.0 */
    return a > b ? a : b;
}

static double julia_min(double a, double b) {
    if (isnan(a)) return a;
    if (isnan(b)) return b;
    if (a == b) return signbit(a) ? a : b;   /* min(-0.0, 0.0) = -0.0 */
    return a < b ? a : b;
}

static double float_at(int dtype, const void *p, int64_t i) {
    return dtype == OD_F32 ? (double)((const float *)p)[i] : ((const double *)p)[i];
}

static void float_put(int dtype, void *p, int64_t i, double v) {
    if (dtype == OD_F32) ((float *)p)[i] = (float)v;
    else ((double *)p)[i] = v;
}

/* integer element i as its raw bits (zero-extended), and as a signed value */
static uint64_t int_bits(int dtype, const void *p, int64_t i) {
    switch (dtype) {
    case OD_U16: case OD_I16: return ((const uint16_t *)p)[i];
    case OD_U32: case OD_I32: return ((const uint32_t *)p)[i];
    default: return ((const uint64_t *)p)[i];
    }
}

static void int_put(int dtype, void *p, int64_t i, uint64_t bits) {
    switch (dtype) {
    case OD_U16: case OD_I16: ((uint16_t *)p)[i] = (uint16_t)bits; break;
    case OD_U32: case OD_I32: ((uint32_t *)p)[i] = (uint32_t)bits; break;
    default: ((uint64_t *)p)[i] = bits; break;
    }
}

/* a < b on raw bits of one integer dtype, by its signedness */
static int int_less(int dtype, uint64_t a, uint64_t b) {
    switch (dtype) {
    case OD_I16: return (int16_t)a < (int16_t)b;
    case OD_I32: return (int32_t)a < (int32_t)b;
    case OD_I64: return (int64_t)a < (int64_t)b;
    default: return a < b;
    }
}

int oracle_accumulate(const void *x, int64_t n, int dtype, int op, int inclusive, const void *init,
                      void *out) {
    if (n < 0 || dtype < 0 || dtype > OD_F64 || op < OA_ADD || op > OA_MIN || !init) return -1;  /* 16-bit floats: not defined here */
    if (n > 0 && (!x || !out)) return -1;
    if (dtype == OD_F32 || dtype == OD_F64) {
        double s = float_at(dtype, init, 0), c = 0.0, plain = s;
#define OA_VALUE (!isfinite(plain) ? plain : (c == 0.0 ? s : s + c))
        for (int64_t i = 0; i < n; ++i) {
            if (!inclusive) float_put(dtype, out, i, OA_VALUE);
            const double v = float_at(dtype, x, i);
            if (op == OA_ADD) {
                const double t = s + v;
                if (fabs(s) >= fabs(v)) c += (s - t) + v;
                else c += (v - t) + s;
                s = t;
                plain = plain + v;
            } else {
                s = op == OA_MAX ? julia_max(s, v) : julia_min(s, v);
                plain = s;
            }
            if (inclusive) float_put(dtype, out, i, OA_VALUE);
        }
#undef OA_VALUE
        return 0;
    }
    uint64_t acc = int_bits(dtype, init, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (!inclusive) int_put(dtype, out, i, acc);
        const uint64_t v = int_bits(dtype, x, i);
        if (op == OA_ADD) acc = acc + v;   /* wraps; int_put keeps the key's width */
        else if (op == OA_MAX) acc = int_less(dtype, acc, v) ? v : acc;
        else acc = int_less(dtype, v, acc) ? v : acc;
        if (dtype == OD_U16 || dtype == OD_I16) acc &= 0xFFFFu;
        else if (dtype == OD_U32 || dtype == OD_I32) acc &= 0xFFFFFFFFu;
        if (inclusive) int_put(dtype, out, i, acc);
    }
    return 0;
}
