"""Counter-based seeded generators for the sort workloads.

Every stream is splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) evaluated at counter positions: the i-th draw of
stream ``seed`` is ``mix64(seed * PHI + (i + 1) * GOLDEN)``.  Because a draw depends
only on (seed, i), any slice of a workload can be regenerated alone, and the
values are identical on every machine and numpy version.

Workloads (the single-device step of the distributed sample sort of Sec. IV-A,
with the dtypes of Sec. IV and the sizes of Sec. IV-C):

* ``uniform_u32``         1,048,576 u32 uniform on [0, 2^32)
* ``uniform_i64``         all 2^64 bit patterns, viewed as int64
* ``normal_f32_special``  N(0,1) float32 with 0.1% NaN (random sign, 22-bit
                          payload) and a disjoint 0.1% of -0.0
* ``dist_f64``            six float64 distributions (uniform, normal,
                          lognormal(0,2), Zipf s=1.2 over 1e6 values, presorted,
                          reverse-sorted)
* ``lognormal_segments``  CSR offsets of 65,536 segments, lognormal lengths with
                          median 2,048 clipped to [1, 2^20]
* ``zipf_mix_u32``        50/50 mix of Zipf(s=1.1, 2^24 ranks, bijectively mixed)
                          and uniform u32
* ``ascending_f64``       keys already in ascending order by construction (a
                          running sum of non-negative steps, a fraction of them
                          zero for runs of equal keys): the sorted input of the
                          binary searches of Sec. II-B, with no sort involved
"""
from __future__ import annotations

import functools

import numpy as np

__all__ = [
    "splitmix64", "u01_f64", "normal_f64", "uniform_u32", "uniform_i64",
    "normal_f32_special", "dist_f64", "F64_DISTS", "lognormal_segments",
    "zipf_mix_u32", "distinct_positions", "fmix32", "special_values",
    "random_keys", "ascending_f64",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_PHI_SEED = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 23


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` draws of stream ``seed`` starting at counter ``start`` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    base = np.uint64((seed * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, count, _CHUNK):
            hi = min(count, lo + _CHUNK)
            ctr = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            out[lo:hi] = _mix64(base + ctr * _GOLDEN)
    return out


def u01_f64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform float64 on [0, 1): the top 53 bits of each draw times 2^-53."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal_f64(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of draws, computed in float64."""
    out = np.empty(count, dtype=np.float64)
    for lo in range(0, count, _CHUNK):
        hi = min(count, lo + _CHUNK)
        z = splitmix64(seed, 2 * (hi - lo), 2 * lo)
        u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
        u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        out[lo:hi] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return out


def uniform_u32(n: int, seed: int = 1) -> np.ndarray:
    return (splitmix64(seed, n) >> np.uint64(32)).astype(np.uint32)


def uniform_i64(n: int, seed: int = 2) -> np.ndarray:
    return splitmix64(seed, n).view(np.int64)


def distinct_positions(n: int, k: int, seed: int) -> np.ndarray:
    """``k`` distinct positions in [0, n), in the order they were first drawn."""
    if k > n:
        raise ValueError("k > n")
    got = np.empty(0, dtype=np.int64)
    start = 0
    while got.size < k:
        want = max(16, int((k - got.size) * 1.1) + 16)
        cand = (splitmix64(seed, want, start) % np.uint64(n)).astype(np.int64)
        start += want
        allc = np.concatenate([got, cand])
        _, first = np.unique(allc, return_index=True)
        got = allc[np.sort(first)]
    return got[:k]


def normal_f32_special(n: int, seed: int = 3, frac: float = 0.001) -> np.ndarray:
    """N(0,1) float32 (Box-Muller in float64, rounded) with round(frac*n) NaNs and
    a disjoint round(frac*n) negative zeros.  Each NaN has a random sign bit and a
    random 22-bit payload under the quiet bit."""
    x = normal_f64(seed, n).astype(np.float32)
    k = int(round(frac * n))
    if k:
        pos = distinct_positions(n, 2 * k, seed + 0x5EED)
        r = splitmix64(seed + 0xBAD, k)
        sign = ((r >> np.uint64(63)) << np.uint64(31)).astype(np.uint32)
        payload = ((r >> np.uint64(8)) & np.uint64(0x3FFFFF)).astype(np.uint32)
        nan_bits = sign | np.uint32(0x7FC00000) | payload
        xb = x.view(np.uint32)
        xb[pos[:k]] = nan_bits
        xb[pos[k:]] = np.uint32(0x80000000)
    return x


F64_DISTS = ("uniform", "normal", "lognormal", "zipf", "presorted", "reversed")


@functools.lru_cache(maxsize=4)
def _zipf_cdf(s: float, nranks: int):
    w = np.arange(1, nranks + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    total = cdf[-1]
    cdf /= total
    return cdf, total


def _zipf_invert(u: np.ndarray, cdf: np.ndarray, total: float, s: float) -> np.ndarray:
    """Exact inverse transform: for each u the index r = #{cdf <= u} (capped at
    nranks-1), i.e. numpy.searchsorted(cdf, u, 'right').  A continuous
    approximation of the harmonic sum (H(k) ~ zeta(s) - k^(1-s)/(s-1)) gives a
    starting index that a few exact neighbour comparisons correct."""
    nranks = cdf.size
    zeta = total + nranks ** (1.0 - s) / (s - 1.0)  # H(K) plus the tail integral
    tail = np.maximum(zeta - u * total, 1e-300) * (s - 1.0)
    r = np.clip(np.floor(tail ** (1.0 / (1.0 - s))).astype(np.int64) - 1, 0, nranks - 1)
    for _ in range(1 << 12):
        up = (r < nranks - 1) & (cdf[r] <= u)
        down = (r > 0) & (cdf[np.maximum(r - 1, 0)] > u)
        if not (up.any() or down.any()):
            break
        r += up.astype(np.int64) - down.astype(np.int64)
    else:  # never expected; keep the definition exact regardless
        r = np.minimum(np.searchsorted(cdf, u, side="right"), nranks - 1)
    return r


def _zipf_ranks(count: int, s: float, nranks: int, seed: int) -> np.ndarray:
    """Zipf(s) ranks in [1, nranks] by inverse transform of a uniform draw."""
    cdf, total = _zipf_cdf(s, nranks)
    out = np.empty(count, dtype=np.int64)
    for lo in range(0, count, _CHUNK):
        hi = min(count, lo + _CHUNK)
        out[lo:hi] = _zipf_invert(u01_f64(seed, hi - lo, lo), cdf, total, s) + 1
    return out


def dist_f64(n: int, dist: str, seed: int) -> np.ndarray:
    if dist == "uniform":
        return u01_f64(seed, n)
    if dist == "normal":
        return normal_f64(seed, n)
    if dist == "lognormal":
        return np.exp(2.0 * normal_f64(seed, n))
    if dist == "zipf":
        table = u01_f64(seed + 0x21F, 1_000_000)
        return table[_zipf_ranks(n, 1.2, 1_000_000, seed) - 1]
    if dist == "presorted":
        return np.sort(u01_f64(seed, n))
    if dist == "reversed":
        return np.sort(u01_f64(seed, n))[::-1].copy()
    raise ValueError(dist)


def lognormal_segments(nseg: int = 65536, seed: int = 20, median: float = 2048.0,
                       max_len: int = 1 << 20) -> np.ndarray:
    """CSR offsets (int64, nseg+1) of segments whose lengths are lognormal with
    the given median and sigma = sqrt(2 ln 2) (mean = 2 x median), rounded and
    clipped to [1, max_len]."""
    sigma = np.sqrt(2.0 * np.log(2.0))
    z = normal_f64(seed, nseg)
    lens = np.clip(np.rint(median * np.exp(sigma * z)), 1, max_len).astype(np.int64)
    off = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


def fmix32(x: np.ndarray) -> np.ndarray:
    """MurmurHash3's 32-bit finaliser: a bijection of uint32."""
    x = x.astype(np.uint32)
    with np.errstate(over="ignore"):
        x = x ^ (x >> np.uint32(16))
        x = x * np.uint32(0x85EBCA6B)
        x = x ^ (x >> np.uint32(13))
        x = x * np.uint32(0xC2B2AE35)
        x = x ^ (x >> np.uint32(16))
    return x


def _zipf_mix_chunk(args):
    lo, hi, seed, s, nranks = args
    cdf, total = _zipf_cdf(s, nranks)
    z = splitmix64(seed, hi - lo, lo)
    coin = (z >> np.uint64(63)).astype(bool)
    u = (z & np.uint64((1 << 53) - 1)).astype(np.float64) * (2.0 ** -53)
    ranks = _zipf_invert(u, cdf, total, s)
    zipf_keys = fmix32(ranks.astype(np.uint32))
    uni = ((z >> np.uint64(16)) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return np.where(coin, zipf_keys, uni)


def zipf_mix_u32(n: int, seed: int = 30, s: float = 1.1, nranks: int = 1 << 24, workers: int = 1) -> np.ndarray:
    """Per key a fair coin picks Zipf(s) over ``nranks`` ranks (rank k maps to
    fmix32(k-1)) or a uniform u32.  ``workers`` > 1 generates chunks in a spawned
    process pool (same values: every chunk depends only on its counter range)."""
    out = np.empty(n, dtype=np.uint32)
    chunk = 1 << 24
    jobs = [(lo, min(n, lo + chunk), seed, s, nranks) for lo in range(0, n, chunk)]
    if workers > 1 and len(jobs) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            for (lo, hi, *_), part in zip(jobs, ex.map(_zipf_mix_chunk, jobs)):
                out[lo:hi] = part
    else:
        for job in jobs:
            out[job[0]:job[1]] = _zipf_mix_chunk(job)
    return out


def special_values(dtype) -> np.ndarray:
    """Edge values of a dtype: extremes, zeros of both signs, infinities, NaNs
    with both signs and distinct payloads, subnormals."""
    dt = np.dtype(dtype)
    if dt.kind in "ui":
        info = np.iinfo(dt)
        vals = [info.min, info.max, 0, 1, info.max - 1, info.min + 1]
        if dt.kind == "i":
            vals += [-1, -2]
        return np.array(vals, dtype=dt)
    if dt == np.float16:
        bits = np.array([0x0000, 0x8000, 0x7C00, 0xFC00, 0x7E00, 0xFE01, 0x7E5A, 0x7C01,
                         0x0001, 0x8001, 0x3C00, 0xBC00, 0x7BFF, 0xFBFF], dtype=np.uint16)
        return bits.view(np.float16)
    if dt == np.float32:
        bits = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000,
                         0xFFC00001, 0x7FC12345, 0x7F800001, 0x00000001, 0x80000001,
                         0x3F800000, 0xBF800000, 0x7F7FFFFF, 0xFF7FFFFF], dtype=np.uint32)
        return bits.view(np.float32)
    if dt == np.float64:
        bits = np.array([0x0, 0x8000000000000000, 0x7FF0000000000000, 0xFFF0000000000000,
                         0x7FF8000000000000, 0xFFF8000000000001, 0x7FF80000DEADBEEF,
                         0x7FF0000000000001, 0x1, 0x8000000000000001, 0x3FF0000000000000,
                         0xBFF0000000000000, 0x7FEFFFFFFFFFFFFF, 0xFFEFFFFFFFFFFFFF],
                        dtype=np.uint64)
        return bits.view(np.float64)
    raise TypeError(dt)


def random_keys(n: int, dtype, seed: int, mode: str = "bits") -> np.ndarray:
    """Test keys of any dtype.

    mode 'bits'  : uniform over all bit patterns (includes NaNs for floats)
    mode 'dups'  : drawn from a small pool (heavy duplicates) mixed with specials
    mode 'narrow': small non-negative integers / a narrow float range (many
                   radix digits constant across all keys)
    """
    dt = np.dtype(dtype)
    raw = splitmix64(seed, n)
    if mode == "bits":
        return raw.astype(np.dtype(f"u{dt.itemsize}")).view(dt) if dt.itemsize < 8 else raw.view(dt)
    if mode == "dups":
        pool = np.concatenate([special_values(dt),
                               random_keys(64, dt, seed + 1, "bits")])
        return pool[(raw % np.uint64(pool.size)).astype(np.int64)]
    if mode == "narrow":
        if dt.kind in "ui":
            return (raw % np.uint64(1000)).astype(dt)
        return (1.0 + (raw >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)).astype(dt)
    raise ValueError(mode)


def ascending_f64(n: int, seed: int = 40, zero_frac: float = 0.25) -> np.ndarray:
    """n float64 keys in ascending order by construction: the running sum of
    steps uniform on [0, 1), a ``zero_frac`` share of them set to 0 (runs of
    equal keys).  A running sum of non-negative float64 terms never decreases,
    so no sort is involved; the values are non-negative and finite."""
    out = np.empty(n, dtype=np.float64)
    acc = 0.0
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        step = u01_f64(seed, hi - lo, lo)
        step[u01_f64(seed + 1, hi - lo, lo) < zero_frac] = 0.0
        np.cumsum(step, out=out[lo:hi])
        out[lo:hi] += acc
        acc = float(out[hi - 1])
    return out
