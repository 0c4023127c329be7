// learned.cuh -- learned-CDF bucketing: the model and its kernels.
//
// The splitter step of the paper's sample sort (Sec. IV-A) draws a key sample
// and turns interpolated histograms of it into splitters.  Here the sample trains
// a small monotone model of the key CDF, F = PL + r:
//   x-hat = min-max normalised coordinate of the key over the sample's range:
//           the radix key (the order-preserving integer image of common.cuh),
//           or, for float keys, a float32 image of the value (negated for a
//           descending sort; NaN after every number) -- whichever of the two
//           overloads buckets less on the sample under the piecewise-linear fit
//           below: the overload of a window of LM_FIT_WINDOW consecutive sample
//           keys is their share of the keys over the share of the CDF the fit
//           gives them; fewer windows above LM_HEAVY wins, then fewer above
//           LM_MODERATE
//           (in radix-key space float keys are roughly logarithmic: heavy tails
//           stay smooth, mass near zero does not; in value space the reverse)
//   PL    = 64-knot piecewise-linear CDF through (xi_j, j/63), xi_j the sample
//           order statistic of rank round(j (m-1) / 63): the sample sort's
//           splitters, interpolated
//   r     = MLP residual 1 -> 16 -> 16 -> 1 (ReLU), trained on (x_i, (i+0.5)/m)
//           with mean squared error by full-batch Adam, deterministic reductions
// F is tabulated at M + 1 points, clamped to [0, 1] and made non-decreasing by a
// running maximum; with B buckets the bucket of a key is
//   floor(B * interp(F table)) clamped into [K[i], K[i+1]],  K[i] = floor(B * T[i])
// which is non-decreasing in the key (each step is monotone; the clamp glues
// table cells).  Sorting stably by bucket and then inside buckets is therefore
// the stable sort, whatever the model learned; the model only decides speed.
#pragma once

#include <float.h>

#include "common.cuh"

namespace ak {

constexpr int LM_KNOTS = 64;
constexpr int LM_HID = 16;
constexpr int LM_PARAMS = 321;  // W1[16] b1[16] W2[16][16] b2[16] w3[16] b3
constexpr int LM_P_W1 = 0, LM_P_B1 = 16, LM_P_W2 = 32, LM_P_B2 = 288, LM_P_W3 = 304, LM_P_B3 = 320;
constexpr int LM_TABLE = 4096;   // table cells M
constexpr int LM_TRAIN = 8192;   // training points T
constexpr int LM_MAX_SAMPLE = 1 << 20;
constexpr int LM_TRAIN_BLOCK = 256;
constexpr int LM_FIT_WINDOW = 64;  // sample keys per window of the coordinate choice
// A window overloaded LM_HEAVY times fills its buckets (half the finish
// capacity each on average) to 16 times the capacity: the plan's overfull mark.
// LM_MODERATE: twice the capacity (one split in the finish).
constexpr float LM_HEAVY = 32.0f;
constexpr float LM_MODERATE = 4.0f;
constexpr int LM_TRAIN_CTAS = LM_TRAIN / LM_TRAIN_BLOCK;  // one point per thread
// r = LM_OUT_SCALE * (b3 + w3 . h2): keeps the residual's steps at the scale of
// the piecewise-linear fit's error while the optimiser takes unit-scale steps
constexpr float LM_OUT_SCALE = 1.0f / 1024.0f;

struct LearnedModel {
  unsigned long long neg_lo;  // ~min radix key of the non-NaN sample (max-reduced)
  unsigned long long hi;      // max radix key of the non-NaN sample
  float inv;                  // 1 / fp32(hi - lo), 0 when hi == lo
  uint32_t m;                 // sample size
  uint32_t bbits, nbuckets;   // log2 B, B
  uint32_t use_plain;         // 1: fall back to the plain radix path
  uint32_t barrier;           // training grid barrier arrivals
  float loss_before, loss_after;
  uint32_t coord;             // 1: float keys use the value coordinate
  uint32_t moderate[2];       // sample windows overloaded above LM_MODERATE: radix, value coordinate
  uint32_t heavy[2];          // sample windows overloaded above LM_HEAVY, per coordinate
  float lo_f, inv_f;          // value coordinate: sample minimum, 1 / sample range
  uint32_t sample_max[2];     // largest run of one bucket in the sorted sample: PL table, PL + MLP table
  uint32_t mlp_used;          // 1: the bucket table holds the MLP residual
  float c_v[LM_KNOTS];        // knots of the value coordinate
  float c[LM_KNOTS];          // PL knots xi_j (x-hat of sample order statistics)
  float params[LM_PARAMS];
  float2 tk[LM_TABLE + 1];    // (T[k], bits of K[k])
};

// ------------------------------------------------------------ device helpers
// Piecewise-linear CDF through the knots (xi_j, j/63): xi = 64 order statistics
// of the sorted sample at ranks round(j (m-1) / 63) (the sample sort's
// splitters, interpolated).  0 below xi_0, 1 from xi_63 on; non-decreasing.
__device__ __forceinline__ float lm_pl(const float *xi, float x) {
  if (!(x >= xi[0])) return 0.f;
  if (x >= xi[LM_KNOTS - 1]) return 1.f;
  int lo = 0, hi = LM_KNOTS - 1;  // invariant: xi[lo] <= x < xi[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (xi[mid] <= x) lo = mid;
    else hi = mid;
  }
  const float f = __fdiv_rn(__fsub_rn(x, xi[lo]), __fsub_rn(xi[hi], xi[lo]));
  return __fdiv_rn(__fadd_rn(float(lo), f), float(LM_KNOTS - 1));
}

// Unscaled residual b3 + w3 . h2(x) (r = LM_OUT_SCALE times this); optionally
// keeps the activations for the backward pass.
__device__ __forceinline__ float lm_mlp(const float *p, float x, float *a1 = nullptr, float *h1o = nullptr,
                                        float *a2 = nullptr, float *h2o = nullptr) {
  float h1[LM_HID];
#pragma unroll
  for (int k = 0; k < LM_HID; ++k) {
    const float a = fmaf(p[LM_P_W1 + k], x, p[LM_P_B1 + k]);
    if (a1) a1[k] = a;
    h1[k] = a > 0.f ? a : 0.f;
    if (h1o) h1o[k] = h1[k];
  }
  float r = p[LM_P_B3];
#pragma unroll
  for (int j = 0; j < LM_HID; ++j) {
    float a = p[LM_P_B2 + j];
#pragma unroll
    for (int k = 0; k < LM_HID; ++k) a = fmaf(p[LM_P_W2 + j * LM_HID + k], h1[k], a);
    if (a2) a2[j] = a;
    const float h = a > 0.f ? a : 0.f;
    if (h2o) h2o[j] = h;
    r = fmaf(p[LM_P_W3 + j], h, r);
  }
  return r;
}

// The bucket of a key is computed by several kernels (histogram and passes) and
// must agree bit for bit: every floating-point step below is an explicitly
// rounded intrinsic, which the compiler neither contracts nor reorders.

// x-hat of a radix key: monotone non-decreasing in r.
template <typename U>
__device__ __forceinline__ float lm_xhat(U r, unsigned long long lo, unsigned long long hi, float inv) {
  const unsigned long long rr = (unsigned long long)r;
  unsigned long long d = rr > lo ? rr - lo : 0ull;
  const unsigned long long span = hi - lo;
  d = d < span ? d : span;
  float x = __fmul_rn(__ull2float_rn(d), inv);
  x = x < 1.f ? x : 1.f;
  return x;
}

// Bucket of x-hat through the monotone table.
__device__ __forceinline__ uint32_t lm_bucket(const float2 *tk, float x, uint32_t nb) {
  const float t = __fmul_rn(x, float(LM_TABLE));
  int i = int(t);
  i = i < LM_TABLE - 1 ? i : LM_TABLE - 1;
  const float f = __fsub_rn(t, float(i));
  const float2 a = tk[i], b = tk[i + 1];
  const float F = fmaf(f, __fsub_rn(b.x, a.x), a.x);  // non-decreasing in f since b.x >= a.x
  uint32_t q = uint32_t(__fmul_rn(F, float(nb)));
  const uint32_t kl = __float_as_uint(a.y), kh = __float_as_uint(b.y);
  q = q < kl ? kl : q;
  q = q > kh ? kh : q;
  return q < nb - 1 ? q : nb - 1;
}

// Value coordinate of a float key from its radix key r (of a sort whose flip is
// `flip`): a float32 image of the value, negated for a descending sort, NaN
// after every number.  A float64 value is narrowed with integer operations
// (exponent rebiased, mantissa truncated, underflow to zero, overflow to the
// largest float), so the image is non-decreasing in r and needs no FP64 unit.
template <typename U>
__device__ __forceinline__ float lm_value_f32(U r, U flip) {
  constexpr U SIGN = U(U(1) << (8 * sizeof(U) - 1));
  const U ra = U(r ^ flip);  // ascending radix key
  const bool desc = flip != U(0);
  if (ra == U(~U(0))) return desc ? -FLT_MAX : FLT_MAX;  // NaN
  const U bits = (ra & SIGN) ? U(ra ^ SIGN) : U(~ra);     // the key's own bits
  uint32_t f;
  if constexpr (sizeof(U) == 8) {
    const uint32_t sgn = uint32_t(uint64_t(bits) >> 63);
    const int e = int((uint64_t(bits) >> 52) & 0x7FFu) - 1023 + 127;
    uint32_t mag;
    if (e <= 0) mag = 0u;                 // below the float range (and zero): 0
    else if (e >= 255) mag = 0x7F7FFFFFu;  // above it (and infinity): FLT_MAX
    else mag = (uint32_t(e) << 23) | uint32_t((uint64_t(bits) >> 29) & 0x7FFFFFu);
    f = (sgn << 31) | mag;
  } else {
    f = uint32_t(bits);
  }
  const float v = __uint_as_float(f);
  return desc ? -v : v;
}

// x-hat of a value coordinate: monotone non-decreasing in v.
__device__ __forceinline__ float lm_xhat_value(float v, float lo, float inv) {
  const float x = __fmul_rn(__fsub_rn(v, lo), inv);
  return x > 0.f ? (x < 1.f ? x : 1.f) : 0.f;  // NaN (inf * 0) -> 0
}

// x-hat of a key from its radix key r.
template <int KIND, typename U>
__device__ __forceinline__ float lm_key_xhat(const LearnedModel *md, U r, U flip) {
  if constexpr (KIND == KIND_FLOAT && sizeof(U) >= 4) {
    if (md->coord) return lm_xhat_value(lm_value_f32(r, flip), md->lo_f, md->inv_f);
  }
  return lm_xhat(r, ~md->neg_lo, md->hi, md->inv);
}

template <int KIND, typename U>
__device__ __forceinline__ uint32_t lm_key_bucket(const LearnedModel *md, U key, U flip) {
  return lm_bucket(md->tk, lm_key_xhat<KIND>(md, radix_key_t<KIND>(key, flip), flip), md->nbuckets);
}

// splitmix64 finaliser on a counter: the sample index stream.
__device__ __forceinline__ unsigned long long lm_mix(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// -------------------------------------------------------- training storage
// Per-point activations are kept in shared memory so that every parameter's
// gradient is a sum over the CTA's points in a fixed order.
struct GradSmem {
  float x[LM_TRAIN_BLOCK], d3[LM_TRAIN_BLOCK], e2[LM_TRAIN_BLOCK];
  float h1[LM_TRAIN_BLOCK][LM_HID + 1];
  float h2[LM_TRAIN_BLOCK][LM_HID + 1];
  float d1[LM_TRAIN_BLOCK][LM_HID + 1];
  float d2[LM_TRAIN_BLOCK][LM_HID + 1];
};

// ------------------------------------------------------------------- sampling
// Gathers the sample's radix keys (as u64) and max-reduces ~r and r over the
// non-NaN sample keys.
template <typename U, int KIND>
__global__ void lm_sample_kernel(const U *keys, int64_t n, U flip, uint32_t m, uint32_t seed,
                                 unsigned long long *sample_r, LearnedModel *md, const uint32_t *gate) {
  if (gate && *gate) return;
  __shared__ unsigned long long s_lo[32], s_hi[32];
  unsigned long long lo_n = 0, hi = 0;  // max of ~r, max of r
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const unsigned long long h = lm_mix((unsigned long long)seed * 0xD1B54A32D192ED03ull + j);
    const U k = keys[int64_t(h % (unsigned long long)n)];
    const U r = radix_key_t<KIND>(k, flip);
    sample_r[j] = (unsigned long long)r;
    bool nonfinite = false;  // NaN and infinities stay out of the range (x-hat clamps them)
    if (KIND == KIND_FLOAT || KIND == KIND_BF16) {
      constexpr U SIGN = U(U(1) << (8 * sizeof(U) - 1));
      nonfinite = U(k & U(~SIGN)) >= float_exp<KIND, U>();
    }
    if (!nonfinite) {
      lo_n = max(lo_n, ~(unsigned long long)r);
      hi = max(hi, (unsigned long long)r);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo_n = max(lo_n, __shfl_xor_sync(0xffffffffu, lo_n, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_lo[w] = lo_n;
    s_hi[w] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < int(blockDim.x >> 5); ++i) {
      lo_n = max(lo_n, s_lo[i]);
      hi = max(hi, s_hi[i]);
    }
    lo_n = max(lo_n, s_lo[0]);
    hi = max(hi, s_hi[0]);
    if (lo_n) atomicMax(&md->neg_lo, lo_n);
    if (hi) atomicMax(&md->hi, hi);
  }
}

// x-hat of every key of the sorted sample in the radix coordinate (xs) and,
// for float keys of `vbytes` (4 or 8; 0: integer keys), the value coordinate
// (xs_v); flip: the sort's flip (all ones when descending).
__global__ void lm_xhat_kernel(const unsigned long long *sample_r, uint32_t m, LearnedModel *md, float *xs,
                               float *xs_v, int vbytes, unsigned long long flip, const uint32_t *gate);

// Windows of LM_FIT_WINDOW consecutive keys of the sorted sample that the PL
// fit overloads above LM_MODERATE and LM_HEAVY, per coordinate (md->moderate,
// md->heavy).
__global__ void lm_fit_error_kernel(const float *xs, const float *xs_v, uint32_t m, LearnedModel *md,
                                    const uint32_t *gate);

// Picks the coordinate with the smaller overload (float keys) and makes its
// knots the model's; sets use_plain at once when the sample shows that the
// plan would fall back.
__global__ void lm_choose_kernel(LearnedModel *md, int has_value, DevHeader *hdr, int64_t n, uint32_t nbuckets,
                                 const uint32_t *gate);

// Knots xi_j = xs[round(j (m-1) / 63)] of an ascending sample.
__global__ void lm_knots_kernel(const float *xs, int64_t m, float *knots, LearnedModel *md, const uint32_t *gate);

// Training: LM_TRAIN_CTAS co-resident CTAs, one training point per thread.
__global__ void lm_train_kernel(const float *xs, const float *xs_v, uint32_t m, LearnedModel *md, float *partials,
                                int steps,
                                float lr, uint32_t init_seed, DevHeader *hdr, uint64_t timeout_ns,
                                const uint32_t *gate);

// Loss and gradient over (x, y) at given params: per-CTA partials, then reduce.
__global__ void lm_grad_partial_kernel(const float *x, const float *y, int64_t m, const float *c,
                                       const float *params, float *partials);
__global__ void lm_grad_reduce_kernel(const float *partials, int nparts, int64_t m, float *grad, float *loss);

// Table T[k] = running max of clamp(F(k/M)), K[k] = min(B-1, floor(B T[k])).
// use_mlp: 0 the piecewise-linear CDF alone, 1 with the MLP residual, 2 as
// md->mlp_used says.
__global__ void lm_table_kernel(LearnedModel *md, int use_mlp, uint32_t nbuckets, uint32_t bbits,
                                const uint32_t *gate);
// Largest number of sorted-sample keys in one bucket under the current table
// (the sample's buckets are non-decreasing): max-reduced into md->sample_max[slot].
__global__ void lm_sample_runs_kernel(const float *xs, const float *xs_v, uint32_t m, LearnedModel *md, int slot,
                                      const uint32_t *gate);
// The MLP residual is kept only when it strictly shrinks the sample's largest
// bucket; records the choice in md->mlp_used and the ak_info.
__global__ void lm_pick_kernel(LearnedModel *md, DevHeader *hdr, const uint32_t *gate);

}  // namespace ak
