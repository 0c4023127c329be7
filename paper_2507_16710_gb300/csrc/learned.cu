// learned.cu -- model kernels of the learned-CDF path (fit, train, tabulate)
// and the C-ABI entry points that expose them for checking.
#include "internal.h"
#include "learned.cuh"
#include "onesweep.cuh"

namespace ak {

__global__ void lm_xhat_kernel(const unsigned long long *sample_r, uint32_t m, LearnedModel *md, float *xs,
                               float *xs_v, int vbytes, unsigned long long flip, const uint32_t *gate) {
  if (gate && *gate) return;
  const unsigned long long lo = ~md->neg_lo, hi = md->hi;
  const bool any = md->hi != 0 || md->neg_lo != 0;
  const unsigned long long l = (any && lo <= hi) ? lo : 0ull, h = (any && lo <= hi) ? hi : 0ull;
  const float inv = (h > l) ? 1.0f / __ull2float_rn(h - l) : 0.0f;
  auto value = [&](unsigned long long r) {
    return vbytes == 8 ? lm_value_f32<uint64_t>(uint64_t(r), uint64_t(flip))
                       : lm_value_f32<uint32_t>(uint32_t(r), uint32_t(flip));
  };
  // value coordinate: range of the finite sample keys
  float lo_f = 0.f, inv_f = 0.f;
  if (vbytes && h > l) {
    lo_f = value(l);
    const float span = __fsub_rn(value(h), lo_f);
    inv_f = (span > 0.f && span <= FLT_MAX) ? __fdiv_rn(1.f, span) : 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    md->neg_lo = ~l;
    md->hi = h;
    md->inv = inv;
    md->lo_f = lo_f;
    md->inv_f = inv_f;
    md->m = m;
  }
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    xs[j] = lm_xhat(sample_r[j], l, h, inv);
    if (vbytes) xs_v[j] = lm_xhat_value(value(sample_r[j]), lo_f, inv_f);
  }
}

__global__ void lm_fit_error_kernel(const float *xs, const float *xs_v, uint32_t m, LearnedModel *md,
                                    const uint32_t *gate) {
  if (gate && *gate) return;
  __shared__ float c[2][LM_KNOTS];
  __shared__ uint32_t s_cnt[2][2];  // [coordinate][moderate, heavy]
  if (threadIdx.x < LM_KNOTS) {
    c[0][threadIdx.x] = md->c[threadIdx.x];
    c[1][threadIdx.x] = md->c_v[threadIdx.x];
  }
  if (threadIdx.x < 4) s_cnt[threadIdx.x >> 1][threadIdx.x & 1] = 0u;
  __syncthreads();
  // overload of a window of k consecutive sample keys: the share of keys it
  // holds over the share of buckets the model gives it
  const uint32_t k = m >= 2 * LM_FIT_WINDOW ? uint32_t(LM_FIT_WINDOW) : (m > 1 ? m / 2 : 1u);
  const float share = float(k) / float(m);
  auto overload = [&](const float *cc, const float *x, uint32_t i) {
    const float d = lm_pl(cc, x[i + k]) - lm_pl(cc, x[i]);
    return d > 0.f ? share / d : FLT_MAX;
  };
  uint32_t n0[2] = {0u, 0u}, n1[2] = {0u, 0u};
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i + k < m; i += gridDim.x * blockDim.x) {
    const float o0 = overload(c[0], xs, i);
    n0[0] += o0 > LM_MODERATE ? 1u : 0u;
    n0[1] += o0 > LM_HEAVY ? 1u : 0u;
    if (xs_v) {
      const float o1 = overload(c[1], xs_v, i);
      n1[0] += o1 > LM_MODERATE ? 1u : 0u;
      n1[1] += o1 > LM_HEAVY ? 1u : 0u;
    }
  }
  for (int q = 0; q < 2; ++q) {
    if (n0[q]) atomicAdd(&s_cnt[0][q], n0[q]);
    if (n1[q]) atomicAdd(&s_cnt[1][q], n1[q]);
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    atomicAdd(&md->moderate[threadIdx.x], s_cnt[threadIdx.x][0]);
    atomicAdd(&md->heavy[threadIdx.x], s_cnt[threadIdx.x][1]);
  }
}

__global__ void lm_choose_kernel(LearnedModel *md, int has_value, DevHeader *hdr, int64_t n, uint32_t nbuckets,
                                 const uint32_t *gate) {
  if (gate && *gate) return;
  // fewer windows far beyond capacity, then fewer moderately overloaded ones;
  // duplicate runs (no model splits them) weigh the same in both coordinates
  const bool value = has_value && (md->heavy[1] < md->heavy[0] ||
                                   (md->heavy[1] == md->heavy[0] && md->moderate[1] < md->moderate[0]));
  if (value && threadIdx.x < LM_KNOTS) md->c[threadIdx.x] = md->c_v[threadIdx.x];
  if (threadIdx.x == 0) {
    md->coord = value ? 1u : 0u;
    // early fallback: more than a quarter of the sample in windows that would
    // overflow their buckets far beyond capacity (the plan's criterion, read
    // off the sample before any pass over the keys)
    const uint32_t heavy = md->heavy[value ? 1 : 0];
    if (uint64_t(heavy) * 4u > uint64_t(md->m)) {
      md->use_plain = 1u;
      hdr->info.path = AK_PATH_RADIX;
      hdr->info.buckets = int32_t(nbuckets);
      hdr->info.overfull_keys = md->m ? int64_t(double(heavy) / double(md->m) * double(n)) : 0;  // estimate
      hdr->info.sample_size = int64_t(md->m);
      hdr->info.coordinate = int64_t(md->coord);
    }
  }
}

__global__ void lm_knots_kernel(const float *xs, int64_t m, float *knots, LearnedModel *md, const uint32_t *gate) {
  if (gate && *gate) return;
  const int j = threadIdx.x;
  if (j >= LM_KNOTS) return;
  const int64_t idx = m > 0 ? (int64_t(j) * (m - 1) + (LM_KNOTS - 1) / 2) / (LM_KNOTS - 1) : 0;
  const float xi = m > 0 ? xs[idx] : 0.f;
  if (knots) knots[j] = xi;
  if (md) md->c[j] = xi;
}

// Forward + backward of one point (valid == false contributes nothing); `scale`
// is dL/dF per unit error (2 / m for the mean squared error).
__device__ __forceinline__ void lm_point(const float *p, const float *c, float x, float y, bool valid, float scale,
                                         GradSmem &g, int t) {
  float a1[LM_HID], h1[LM_HID], a2[LM_HID], h2[LM_HID];
  const float r = LM_OUT_SCALE * lm_mlp(p, x, a1, h1, a2, h2);
  const float e = valid ? (lm_pl(c, x) + r - y) : 0.f;
  const float d3 = scale * e * LM_OUT_SCALE;  // dL / d(b3 + w3 . h2)
  g.x[t] = x;
  g.d3[t] = d3;
  g.e2[t] = e * e;
  float d2[LM_HID];
#pragma unroll
  for (int j = 0; j < LM_HID; ++j) {
    d2[j] = a2[j] > 0.f ? d3 * p[LM_P_W3 + j] : 0.f;
    g.d2[t][j] = d2[j];
    g.h2[t][j] = h2[j];
  }
#pragma unroll
  for (int k = 0; k < LM_HID; ++k) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < LM_HID; ++j) s = fmaf(d2[j], p[LM_P_W2 + j * LM_HID + k], s);
    g.d1[t][k] = a1[k] > 0.f ? s : 0.f;
    g.h1[t][k] = h1[k];
  }
}

// Gradient of parameter q summed over the CTA's points: four interleaved
// accumulators (point t goes to accumulator t % 4), combined in a fixed order,
// so the result is deterministic and the dependent chain is a quarter as long.
template <typename F>
__device__ __forceinline__ float lm_sum4(F term) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  for (int t = 0; t < LM_TRAIN_BLOCK; t += 4) {
    s0 += term(t);
    s1 += term(t + 1);
    s2 += term(t + 2);
    s3 += term(t + 3);
  }
  return (s0 + s1) + (s2 + s3);
}

__device__ __forceinline__ float lm_param_grad(const GradSmem &g, int q) {
  if (q < LM_P_B1) return lm_sum4([&](int t) { return g.d1[t][q] * g.x[t]; });
  if (q < LM_P_W2) return lm_sum4([&](int t) { return g.d1[t][q - LM_P_B1]; });
  if (q < LM_P_B2) {
    const int j = (q - LM_P_W2) / LM_HID, k = (q - LM_P_W2) % LM_HID;
    return lm_sum4([&](int t) { return g.d2[t][j] * g.h1[t][k]; });
  }
  if (q < LM_P_W3) return lm_sum4([&](int t) { return g.d2[t][q - LM_P_B2]; });
  if (q < LM_P_B3) return lm_sum4([&](int t) { return g.d3[t] * g.h2[t][q - LM_P_W3]; });
  if (q == LM_P_B3) return lm_sum4([&](int t) { return g.d3[t]; });
  return lm_sum4([&](int t) { return g.e2[t]; });  // q == LM_PARAMS: the loss numerator
}

constexpr int LM_SLOTS = LM_PARAMS + 1;  // gradients + loss numerator

// Uniform in [-1, 1) from (seed, index): initialisation stream.
__device__ __forceinline__ float lm_unif(uint32_t seed, int i) {
  return float(int64_t(lm_mix(((unsigned long long)seed << 32) ^ (unsigned long long)(i + 1)) >> 11)) *
             (2.0f / 9007199254740992.0f) -
         1.0f;
}

// Hinge-basis start: unit k of layer 1 bends at x = (k + 0.5) / 16; the
// output layer starts at zero, so F = PL at step 0.
__device__ __forceinline__ float lm_init_param(uint32_t seed, int q) {
  if (q < LM_P_B1) return 4.0f + 0.5f * lm_unif(seed, q);
  if (q < LM_P_W2) {
    const int k = q - LM_P_B1;
    return -(4.0f + 0.5f * lm_unif(seed, k)) * (float(k) + 0.5f) / float(LM_HID);
  }
  if (q < LM_P_B2) return 0.25f * lm_unif(seed, q);
  if (q < LM_P_W3) return 0.05f * lm_unif(seed, q);
  return 0.0f;
}

__global__ void __launch_bounds__(LM_TRAIN_BLOCK) lm_train_kernel(const float *xs, const float *xs_v, uint32_t m,
                                                                  LearnedModel *md, float *partials, int steps,
                                                                  float lr,
                                                                  uint32_t init_seed, DevHeader *hdr,
                                                                  uint64_t timeout_ns, const uint32_t *gate) {
  if (gate && *gate) return;
  extern __shared__ __align__(16) uint8_t lm_smem[];
  GradSmem &g = *reinterpret_cast<GradSmem *>(lm_smem);
  __shared__ float p[LM_PARAMS], am[LM_PARAMS], av[LM_PARAMS], c[LM_KNOTS];
  __shared__ float s_loss;
  __shared__ int s_abort;
  const int t = threadIdx.x;
  const int G = gridDim.x;
  for (int q = t; q < LM_PARAMS; q += LM_TRAIN_BLOCK) {
    p[q] = lm_init_param(init_seed, q);
    am[q] = 0.f;
    av[q] = 0.f;
  }
  if (t < LM_KNOTS) c[t] = md->c[t];
  if (t == 0) s_abort = 0;
  // training points: T_eff evenly spaced order statistics of the sorted sample
  const int64_t teff = m < LM_TRAIN ? int64_t(m) : int64_t(LM_TRAIN);
  const int64_t gi = int64_t(blockIdx.x) * LM_TRAIN_BLOCK + t;
  const bool valid = gi < teff;
  float x = 0.f, y = 0.f;
  if (valid) {
    const int64_t idx = int64_t((double(gi) + 0.5) * double(m) / double(teff));
    x = (md->coord && xs_v) ? xs_v[idx] : xs[idx];  // the coordinate chosen on the sample
    y = (float(idx) + 0.5f) / float(m);
  }
  const float scale = teff > 0 ? 2.0f / float(teff) : 0.f;
  __syncthreads();
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float b1t = 1.f, b2t = 1.f;
  for (int s = 0; s <= steps; ++s) {
    lm_point(p, c, x, y, valid, scale, g, t);
    __syncthreads();
    float *mine = partials + (size_t(s & 1) * G + blockIdx.x) * LM_SLOTS;
    for (int q = t; q < LM_SLOTS; q += LM_TRAIN_BLOCK) mine[q] = lm_param_grad(g, q);
    // grid barrier s (bounded)
    __threadfence();
    __syncthreads();
    if (t == 0) {
      atomicAdd(&md->barrier, 1u);
      const uint32_t want = uint32_t(s + 1) * uint32_t(G);
      const uint64_t t0 = globaltimer_ns();
      while (ld_relaxed(&md->barrier) < want) {
        __nanosleep(32);
        if (globaltimer_ns() - t0 > timeout_ns) {
          set_error(hdr, AK_ERR_TIMEOUT);
          s_abort = 1;
          break;
        }
      }
      __threadfence();
    }
    __syncthreads();
    if (s_abort) break;
    const float *all = partials + size_t(s & 1) * G * LM_SLOTS;
    b1t *= b1;
    b2t *= b2;
    for (int q = t; q < LM_SLOTS; q += LM_TRAIN_BLOCK) {
      float tot = 0.f;  // fixed order over CTAs; L2 loads (other SMs wrote them)
      for (int k = 0; k < G; ++k) tot += __ldcg(all + size_t(k) * LM_SLOTS + q);
      if (q == LM_PARAMS) {
        s_loss = teff > 0 ? tot / float(teff) : 0.f;
      } else if (s < steps) {  // Adam (Kingma & Ba), bias-corrected
        am[q] = b1 * am[q] + (1.f - b1) * tot;
        av[q] = b2 * av[q] + (1.f - b2) * tot * tot;
        const float mh = am[q] / (1.f - b1t), vh = av[q] / (1.f - b2t);
        p[q] -= lr * mh / (sqrtf(vh) + eps);
      }
    }
    __syncthreads();
    if (blockIdx.x == 0 && t == 0) {
      if (s == 0) md->loss_before = s_loss;
      if (s == steps) md->loss_after = s_loss;
    }
  }
  if (blockIdx.x == 0)
    for (int q = t; q < LM_PARAMS; q += LM_TRAIN_BLOCK) md->params[q] = p[q];
}

__global__ void __launch_bounds__(LM_TRAIN_BLOCK) lm_grad_partial_kernel(const float *x, const float *y, int64_t m,
                                                                         const float *c, const float *params,
                                                                         float *partials) {
  extern __shared__ __align__(16) uint8_t lm_smem[];
  GradSmem &g = *reinterpret_cast<GradSmem *>(lm_smem);
  __shared__ float p[LM_PARAMS], cc[LM_KNOTS];
  const int t = threadIdx.x;
  for (int q = t; q < LM_PARAMS; q += LM_TRAIN_BLOCK) p[q] = params[q];
  if (t < LM_KNOTS) cc[t] = c[t];
  __syncthreads();
  const int64_t i = int64_t(blockIdx.x) * LM_TRAIN_BLOCK + t;
  const bool valid = i < m;
  lm_point(p, cc, valid ? x[i] : 0.f, valid ? y[i] : 0.f, valid, m > 0 ? 2.0f / float(m) : 0.f, g, t);
  __syncthreads();
  for (int q = t; q < LM_SLOTS; q += LM_TRAIN_BLOCK) partials[size_t(blockIdx.x) * LM_SLOTS + q] = lm_param_grad(g, q);
}

__global__ void lm_grad_reduce_kernel(const float *partials, int nparts, int64_t m, float *grad, float *loss) {
  for (int q = threadIdx.x; q < LM_SLOTS; q += blockDim.x) {
    float tot = 0.f;
    for (int k = 0; k < nparts; ++k) tot += partials[size_t(k) * LM_SLOTS + q];
    if (q < LM_PARAMS) grad[q] = tot;
    else *loss = m > 0 ? tot / float(m) : 0.f;
  }
}

__global__ void __launch_bounds__(1024) lm_table_kernel(LearnedModel *md, int use_mlp, uint32_t nbuckets,
                                                        uint32_t bbits, const uint32_t *gate) {
  if (gate && *gate) return;
  if (threadIdx.x == 0) {
    md->nbuckets = nbuckets;
    md->bbits = bbits;
  }
  if (use_mlp == 2) use_mlp = int(md->mlp_used);
  __shared__ float p[LM_PARAMS], c[LM_KNOTS];
  __shared__ float run[1024];
  constexpr int PER = (LM_TABLE + 1 + 1023) / 1024;  // values per thread (5)
  const int t = threadIdx.x;
  for (int q = t; q < LM_PARAMS; q += 1024) p[q] = md->params[q];
  if (t < LM_KNOTS) c[t] = md->c[t];
  __syncthreads();
  float v[PER];
  float mx = 0.f;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = t * PER + i;
    float F = 0.f;
    if (k <= LM_TABLE) {
      const float u = float(k) / float(LM_TABLE);
      F = lm_pl(c, u) + (use_mlp ? LM_OUT_SCALE * lm_mlp(p, u) : 0.f);
      F = F > 0.f ? F : 0.f;  // NaN-safe clamp into [0, 1]
      F = F < 1.f ? F : 1.f;
    }
    mx = F > mx ? F : mx;
    v[i] = mx;  // running max inside the thread's run
  }
  run[t] = mx;
  __syncthreads();
  // exclusive running max over the thread runs (Hillis-Steele on 1024 values)
  for (int o = 1; o < 1024; o <<= 1) {
    const float other = t >= o ? run[t - o] : 0.f;
    __syncthreads();
    run[t] = run[t] > other ? run[t] : other;
    __syncthreads();
  }
  const float before = t > 0 ? run[t - 1] : 0.f;
  const uint32_t nb = nbuckets;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = t * PER + i;
    if (k <= LM_TABLE) {
      const float T = v[i] > before ? v[i] : before;
      uint32_t K = uint32_t(__fmul_rn(T, float(nb)));
      K = K < nb - 1 ? K : nb - 1;
      md->tk[k] = make_float2(T, __uint_as_float(K));
    }
  }
}

__global__ void lm_sample_runs_kernel(const float *xs, const float *xs_v, uint32_t m, LearnedModel *md, int slot,
                                      const uint32_t *gate) {
  if (gate && *gate) return;
  const float *x = (md->coord && xs_v) ? xs_v : xs;  // the model's coordinate of the sorted sample
  const uint32_t nb = md->nbuckets;
  uint32_t best = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const uint32_t b = lm_bucket(md->tk, x[i], nb);
    if (i + 1 < m && lm_bucket(md->tk, x[i + 1], nb) == b) continue;  // not the last key of its run
    uint32_t lo = 0, hi = i;  // first index of the run: the first j with bucket(x[j]) == b
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (lm_bucket(md->tk, x[mid], nb) < b) lo = mid + 1;
      else hi = mid;
    }
    const uint32_t len = i - lo + 1;
    best = len > best ? len : best;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t other = __shfl_xor_sync(0xffffffffu, best, o);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(&md->sample_max[slot], best);
}

__global__ void lm_pick_kernel(LearnedModel *md, DevHeader *hdr, const uint32_t *gate) {
  if (gate && *gate) return;
  const uint32_t use = md->sample_max[1] != 0 && md->sample_max[1] < md->sample_max[0] ? 1u : 0u;
  md->mlp_used = use;
  hdr->info.mlp_used = int32_t(use);
  hdr->info.sample_max_pl = int64_t(md->sample_max[0]);
  hdr->info.sample_max_mlp = int64_t(md->sample_max[1]);
}

__global__ void __launch_bounds__(1024) lm_plan_kernel(const uint32_t *counts, int64_t n, LearnedModel *md,
                                                       RadixPlan *plan, DevHeader *hdr, int64_t *seg_off,
                                                       int64_t cap) {
  if (md->use_plain) return;
  constexpr int NWARP = 1024 / 32;
  __shared__ unsigned long long d0[RADIX], d1[RADIX], scr[33];
  __shared__ unsigned long long w_sum[NWARP], w_over[NWARP], w_max[NWARP];
  __shared__ int triv[2];
  const uint32_t nb = md->nbuckets, bb = md->bbits;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (t < RADIX) {
    d0[t] = 0ull;
    d1[t] = 0ull;
  }
  if (t < 2) triv[t] = 0;
  __syncthreads();
  // each warp owns a contiguous chunk of buckets and walks it 32 at a time
  // (coalesced loads, shuffle scans); pass 1 sums, pass 2 writes offsets
  const uint32_t chunk = (nb + NWARP - 1) / NWARP;
  const uint32_t c0 = uint32_t(warp) * chunk, c1 = (c0 + chunk) < nb ? (c0 + chunk) : nb;
  unsigned long long sum = 0, over = 0, mx = 0;
  for (uint32_t b0 = c0; b0 < c1; b0 += 32) {
    const uint32_t b = b0 + lane;
    const unsigned long long c = b < c1 ? counts[b] : 0ull;
    sum += c;
    if (int64_t(c) > 16 * cap) over += c;  // far above capacity: more than one split away
    mx = c > mx ? c : mx;
    if (c) atomicAdd(&d0[b & (RADIX - 1)], c);  // 32 consecutive buckets: 32 distinct digits
    if (bb > RADIX_BITS) {
      // high-byte digit: the bucket count is a power of two >= 512, so chunks
      // (nb / 32 >= 16 buckets) and their 32-bucket groups are aligned and never
      // straddle a 256-bucket block: one digit per group
      unsigned long long hi = c;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hi += __shfl_xor_sync(0xffffffffu, hi, o);
      if (lane == 0 && hi) atomicAdd(&d1[b0 >> RADIX_BITS], hi);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    over += __shfl_xor_sync(0xffffffffu, over, o);
    const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
  }
  if (lane == 0) {
    w_sum[warp] = sum;
    w_over[warp] = over;
    w_max[warp] = mx;
  }
  __syncthreads();
  unsigned long long base = 0, s_over = 0, s_max = 0;
  for (int w = 0; w < NWARP; ++w) {
    if (w < warp) base += w_sum[w];
    s_over += w_over[w];
    s_max = w_max[w] > s_max ? w_max[w] : s_max;
  }
  // offsets: warp-level exclusive scans over the chunk, 32 buckets at a time
  unsigned long long run = base;
  for (uint32_t b0 = c0; b0 < c1; b0 += 32) {
    const uint32_t b = b0 + lane;
    const unsigned long long c = b < c1 ? counts[b] : 0ull;
    unsigned long long inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (b < c1) seg_off[b] = int64_t(run + inc - c);
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (t == 0) seg_off[nb] = n;
  __syncthreads();
  unsigned long long tot;
  const int passes = int((bb + RADIX_BITS - 1) / RADIX_BITS);
  for (int p = 0; p < passes; ++p) {
    const unsigned long long c = t < RADIX ? (p == 0 ? d0[t] : d1[t]) : 0ull;
    if (t < RADIX && c == (unsigned long long)n) triv[p] = 1;
    const unsigned long long ex = block_exclusive_scan<1024>(c, scr, &tot);
    if (t < RADIX) plan->bin_off[p][t] = ex;
  }
  __syncthreads();
  if (t == 0) {
    uint32_t m = 0;
    for (int p = 0; p < MAX_PASSES; ++p) plan->q[p] = (p < passes && !triv[p]) ? m++ : INACTIVE;
    plan->m = m;
    // fallback when more than a quarter of the keys sit in buckets above capacity
    const uint32_t plain = (s_over * 4ull > (unsigned long long)n) ? 1u : 0u;
    md->use_plain = plain;
    hdr->info.path = plain ? AK_PATH_RADIX : AK_PATH_LEARNED;
    hdr->info.radix_passes = int32_t(m);
    hdr->info.buckets = int32_t(nb);
    hdr->info.overfull_keys = int64_t(s_over);
    hdr->info.max_bucket = int64_t(s_max);
    hdr->info.loss_before = md->loss_before;
    hdr->info.loss_after = md->loss_after;
    hdr->info.sample_size = int64_t(md->m);
    hdr->info.coordinate = int64_t(md->coord);
  }
}

}  // namespace ak

using namespace ak;

extern "C" {

ak_status ak_learned_knots(const float *d_xs, int64_t m, float *d_knots, ak_stream_t stream) {
  if (m <= 0 || !d_xs || !d_knots) return AK_ERR_INVALID_ARG;
  lm_knots_kernel<<<1, LM_KNOTS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(d_xs, m, d_knots, nullptr, nullptr);
  return cudaGetLastError() == cudaSuccess ? AK_OK : AK_ERR_CUDA;
}

size_t ak_learned_grad_temp_bytes(int64_t m) {
  const int64_t blocks = m > 0 ? (m + LM_TRAIN_BLOCK - 1) / LM_TRAIN_BLOCK : 1;
  return size_t(blocks) * LM_SLOTS * sizeof(float) + 256;
}

ak_status ak_learned_loss_grad(const float *d_x, const float *d_y, int64_t m, const float *d_c,
                               const float *d_params, float *d_grad, float *d_loss, void *d_temp, size_t temp_bytes,
                               ak_stream_t stream) {
  if (m < 0 || !d_c || !d_params || !d_grad || !d_loss || (m > 0 && (!d_x || !d_y))) return AK_ERR_INVALID_ARG;
  if (!d_temp || temp_bytes < ak_learned_grad_temp_bytes(m)) return AK_ERR_WORKSPACE_TOO_SMALL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = int(m > 0 ? (m + LM_TRAIN_BLOCK - 1) / LM_TRAIN_BLOCK : 1);
  const int smem = int(sizeof(GradSmem));
  if (cudaFuncSetAttribute(lm_grad_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return AK_ERR_CUDA;
  float *parts = static_cast<float *>(d_temp);
  lm_grad_partial_kernel<<<blocks, LM_TRAIN_BLOCK, smem, st>>>(d_x, d_y, m, d_c, d_params, parts);
  lm_grad_reduce_kernel<<<1, 352, 0, st>>>(parts, blocks, m, d_grad, d_loss);
  return cudaGetLastError() == cudaSuccess ? AK_OK : AK_ERR_CUDA;
}

}  // extern "C"

namespace ak {
size_t learned_model_bytes() { return sizeof(LearnedModel); }
size_t learned_partials_bytes() { return size_t(2) * LM_TRAIN_CTAS * LM_SLOTS * sizeof(float); }
}  // namespace ak
