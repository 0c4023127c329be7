"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: Julia's documented
isless facts (golden files), the brute-force definition of a stable sort,
Python's stable Timsort, a counting sort, permutation closed forms and
invariants.  A dropped NaN rule, a flipped sign test or an unstable merge fails
at least one of these.
"""
import itertools
import math
import os
import struct

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DTYPES = [np.uint16, np.int16, np.uint32, np.int32, np.uint64, np.int64, np.float32, np.float64]


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("name,ut,ft", [("isless_f64.txt", np.uint64, np.float64),
                                        ("isless_f32.txt", np.uint32, np.float32)])
def test_isless_golden(name, ut, ft):
    rows = _rows(name)
    a = np.array([int(r[0], 16) for r in rows], dtype=ut).view(ft)
    b = np.array([int(r[1], 16) for r in rows], dtype=ut).view(ft)
    want = np.array([r[2] == "1" for r in rows])
    assert np.array_equal(oracle.isless(a, b), want)


def test_sorted_special_golden():
    rows = _rows("sorted_special_f64.txt")
    x, asc, desc = [np.array([int(t, 16) for t in r], dtype=np.uint64).view(np.float64) for r in rows]
    assert np.array_equal(oracle.sort(x, "ascending").view(np.uint64), asc.view(np.uint64))
    assert np.array_equal(oracle.sort(x, "descending").view(np.uint64), desc.view(np.uint64))


def _py_key(v):
    """Sort key for Python's sorted() giving Julia isless order (independent of the oracle)."""
    if isinstance(v, float):
        if math.isnan(v):
            return (1, 0.0, 0)
        return (0, v, 0 if math.copysign(1.0, v) < 0 else 1)
    return (0, v, 0)


def _is_stable_sorted(keys, perm, desc):
    """Brute-force definition: for every i < j, key[p_i] comes strictly before
    key[p_j], or they are equivalent and p_i < p_j."""
    n = len(perm)
    for i in range(n):
        for j in range(i + 1, n):
            a, b = keys[perm[i]:perm[i] + 1], keys[perm[j]:perm[j] + 1]
            lt_ab = oracle.isless(b, a)[0] if desc else oracle.isless(a, b)[0]
            lt_ba = oracle.isless(a, b)[0] if desc else oracle.isless(b, a)[0]
            if lt_ab:
                continue
            if not lt_ba and perm[i] < perm[j]:
                continue
            return False
    return True


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.int32, np.uint16])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 6])
@pytest.mark.parametrize("desc", [False, True])
def test_brute_force_unique_stable_permutation(dtype, n, desc):
    pool = synth.special_values(dtype)
    rng_idx = synth.splitmix64(100 + n, n) % np.uint64(pool.size)
    keys = pool[rng_idx.astype(np.int64)]
    if n >= 3:
        keys[1] = keys[0]  # force a tie so stability matters
    survivors = [p for p in itertools.permutations(range(n)) if _is_stable_sorted(keys, p, desc)]
    assert len(survivors) == 1
    got = oracle.sortperm(keys, "descending" if desc else "ascending")
    assert tuple(got.tolist()) == survivors[0]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("mode", ["bits", "dups", "narrow"])
@pytest.mark.parametrize("desc", [False, True])
def test_matches_python_timsort(dtype, mode, desc):
    keys = synth.random_keys(3000, dtype, seed=7, mode=mode)
    pyvals = [float(v) if np.dtype(dtype).kind == "f" else int(v) for v in keys]
    want = sorted(range(keys.size), key=lambda i: _py_key(pyvals[i]), reverse=desc)
    got = oracle.sortperm(keys, "descending" if desc else "ascending")
    assert np.array_equal(got, np.array(want))


@pytest.mark.parametrize("dtype", [np.uint16, np.int16])
@pytest.mark.parametrize("desc", [False, True])
def test_counting_sort_16bit(dtype, desc):
    """A counting sort (a different algorithm) on 16-bit keys."""
    keys = synth.random_keys(20000, dtype, seed=11, mode="dups")
    v = keys.astype(np.int64)
    lo = int(v.min())
    counts = np.bincount(v - lo, minlength=int(v.max()) - lo + 1)
    if desc:
        counts_rev = counts[::-1]
        starts = np.concatenate([[0], np.cumsum(counts_rev)[:-1]])[::-1]
    else:
        starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    perm = np.empty(keys.size, dtype=np.int64)
    nxt = starts.copy()
    for i, key in enumerate(v - lo):
        perm[nxt[key]] = i
        nxt[key] += 1
    assert np.array_equal(oracle.sortperm(keys, "descending" if desc else "ascending"), perm)


@pytest.mark.parametrize("dtype", [np.int64, np.uint32, np.int16])
def test_numpy_stable_argsort_on_ints(dtype):
    keys = synth.random_keys(50000, dtype, seed=5, mode="dups")
    assert np.array_equal(oracle.sortperm(keys), np.argsort(keys, kind="stable"))


def test_inverse_permutation_closed_form():
    n = 10007
    pi = np.argsort(synth.splitmix64(9, n), kind="stable")   # a permutation
    keys = np.empty(n, dtype=np.int64)
    keys[pi] = np.arange(n)                                  # keys = pi^-1 ... shuffled iota
    p = oracle.sortperm(keys)
    assert np.array_equal(keys[p], np.arange(n))
    assert np.array_equal(p, pi)


def test_presorted_and_reversed():
    x = np.sort(synth.u01_f64(4, 5000))
    assert np.array_equal(oracle.sortperm(x), np.arange(x.size))
    assert np.array_equal(oracle.sortperm(x[::-1].copy()), np.arange(x.size)[::-1])
    assert np.array_equal(oracle.sortperm(x, "descending"), np.arange(x.size)[::-1])


def test_descending_is_not_reverse_of_ascending_on_ties():
    keys = np.array([2, 1, 2, 1], dtype=np.int32)
    assert oracle.sortperm(keys, "descending").tolist() == [0, 2, 1, 3]
    assert oracle.sortperm(keys, "ascending").tolist() == [1, 3, 0, 2]


def test_nan_payloads_keep_input_order():
    bits = np.array([0x7FC00003, 0x3F800000, 0xFFC00001, 0x7FC00002, 0x80000000, 0x00000000],
                    dtype=np.uint32)
    x = bits.view(np.float32)
    out = oracle.sort(x).view(np.uint32)
    assert out.tolist() == [0x80000000, 0x00000000, 0x3F800000, 0x7FC00003, 0xFFC00001, 0x7FC00002]
    out = oracle.sort(x, "descending").view(np.uint32)
    assert out.tolist() == [0x7FC00003, 0xFFC00001, 0x7FC00002, 0x3F800000, 0x00000000, 0x80000000]


@pytest.mark.parametrize("dtype", [np.float32, np.int64])
def test_threaded_equals_single(dtype):
    keys = synth.random_keys(200003, dtype, seed=3, mode="dups")
    for order in ("ascending", "descending"):
        assert np.array_equal(oracle.sortperm(keys, order), oracle.sortperm(keys, order, threads=7))


def test_pairs_and_gather_move_raw_bits():
    keys = synth.normal_f32_special(10000, seed=8, frac=0.01)
    vals = np.arange(keys.size, dtype=np.uint32)
    k, v = oracle.sort_pairs(keys, vals)
    assert np.array_equal(keys.view(np.uint32)[v], k.view(np.uint32))
    # the multiset of raw bits is unchanged
    assert np.array_equal(np.sort(k.view(np.uint32)), np.sort(keys.view(np.uint32)))


def test_segmented_equals_per_segment_sort():
    off = synth.lognormal_segments(200, seed=20, median=50.0, max_len=2000)
    n = int(off[-1])
    keys = synth.random_keys(n, np.float32, seed=21, mode="dups")
    got = oracle.sortperm_segmented(keys, off)
    for s in range(off.size - 1):
        a, b = int(off[s]), int(off[s + 1])
        assert np.array_equal(got[a:b], a + oracle.sortperm(keys[a:b]))


@pytest.mark.parametrize("desc", [False, True])
def test_segmented_matches_numpy_per_segment(desc):
    """Independent of the merge sort: per segment, numpy's stable argsort of
    unsigned keys (descending: of their bitwise complement, which reverses the
    order and keeps ties in input order); equal keys on both sides of a segment
    boundary must not mix."""
    off = synth.lognormal_segments(300, seed=22, median=40.0, max_len=3000)
    n = int(off[-1])
    keys = (synth.splitmix64(23, n) % np.uint64(7)).astype(np.uint32)  # heavy ties everywhere
    got = oracle.sortperm_segmented(keys, off, "descending" if desc else "ascending")
    for s in range(off.size - 1):
        a, b = int(off[s]), int(off[s + 1])
        seg = ~keys[a:b] if desc else keys[a:b]
        assert np.array_equal(got[a:b], a + np.argsort(seg, kind="stable"))


@pytest.mark.parametrize("dtype", [np.uint16, np.uint32, np.uint64])
def test_descending_matches_numpy_on_complement(dtype):
    """Descending stable order of unsigned keys is numpy's stable argsort of ~k."""
    keys = synth.random_keys(40000, dtype, seed=6, mode="dups")
    assert np.array_equal(oracle.sortperm(keys, "descending"), np.argsort(~keys, kind="stable"))


def test_segmented_rejects_bad_offsets():
    keys = np.arange(10, dtype=np.int32)
    with pytest.raises(RuntimeError):
        oracle.sortperm_segmented(keys, np.array([0, 6, 4, 10]))
    with pytest.raises(RuntimeError):
        oracle.sortperm_segmented(keys, np.array([0, 4, 9]))


def test_generators_are_reproducible_and_shaped():
    a = synth.normal_f32_special(100000, seed=3)
    b = synth.normal_f32_special(100000, seed=3)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert np.isnan(a).sum() == 100
    assert (a.view(np.uint32) == 0x80000000).sum() == 100
    x = synth.normal_f64(3, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    off = synth.lognormal_segments()
    lens = np.diff(off)
    assert lens.size == 65536 and lens.min() >= 1 and lens.max() <= 1 << 20
    assert abs(np.median(lens) - 2048) < 100
    z = synth.zipf_mix_u32(1 << 20, seed=30)
    top = synth.fmix32(np.array([0], dtype=np.uint32))[0]
    frac = (z == top).mean()
    assert 0.04 < frac < 0.08   # ~5.75% of keys equal the top rank
    # ascending by construction, across chunk boundaries, with ~25% equal neighbours
    asc = synth.ascending_f64((1 << 23) + 1000, seed=40)
    assert np.array_equal(asc, synth.ascending_f64((1 << 23) + 1000, seed=40))
    assert np.all(np.diff(asc) >= 0) and np.isfinite(asc).all() and asc[0] >= 0
    assert 0.24 < (np.diff(asc) == 0).mean() < 0.26


# ------------------------------------------------------------ binary search
# Sec. II-B: searchsortedfirst / searchsortedlast (0-based here: Julia's value
# minus one).  Pinned against the brute-force count that defines them, numpy's
# searchsorted where isless is plain <, and hand-derived special values.

def _order_before(a, b, desc):
    """a comes strictly before b in the order (isless, or reversed isless)."""
    return oracle.isless(b, a) if desc else oracle.isless(a, b)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("desc", [False, True])
def test_searchsorted_brute_force_count(dtype, desc):
    order = "descending" if desc else "ascending"
    keys = np.concatenate([synth.random_keys(150, dtype, seed=71, mode="dups"), synth.special_values(dtype)])
    v = oracle.sort(keys, order)
    x = np.concatenate([synth.random_keys(60, dtype, seed=72, mode="dups"), synth.random_keys(20, dtype, seed=73),
                        synth.special_values(dtype)])
    first, last = oracle.searchsorted(v, x, "first", order), oracle.searchsorted(v, x, "last", order)
    for i in range(x.size):
        xi = np.full(v.size, x[i], dtype=v.dtype)
        n_before = int(np.count_nonzero(_order_before(v, xi, desc)))       # v[j] before x
        n_not_after = int(np.count_nonzero(~_order_before(xi, v, desc)))  # x not before v[j]
        assert first[i] == n_before, (i, x[i])
        assert last[i] == n_not_after - 1, (i, x[i])


@pytest.mark.parametrize("dtype", [np.uint32, np.int64, np.float64, np.int16])
def test_searchsorted_matches_numpy(dtype):
    """Without NaN or -0.0, isless is <: numpy's searchsorted gives both sides;
    a descending v is the ascending one reversed (counts from the other end)."""
    raw = synth.random_keys(5000, dtype, seed=74, mode="narrow")
    if np.dtype(dtype).kind == "f":
        raw = np.abs(raw)
    asc = np.sort(raw, kind="stable")
    x = np.concatenate([raw[:700], synth.random_keys(300, dtype, seed=75, mode="narrow")])
    if np.dtype(dtype).kind == "f":
        x = np.abs(x)
    n = asc.size
    assert np.array_equal(oracle.searchsorted(asc, x, "first"), np.searchsorted(asc, x, "left"))
    assert np.array_equal(oracle.searchsorted(asc, x, "last"), np.searchsorted(asc, x, "right") - 1)
    desc = asc[::-1].copy()
    assert np.array_equal(oracle.searchsorted(desc, x, "first", "descending"), n - np.searchsorted(asc, x, "right"))
    assert np.array_equal(oracle.searchsorted(desc, x, "last", "descending"),
                          n - np.searchsorted(asc, x, "left") - 1)


def test_searchsorted_special_values_by_hand():
    """Worked from Julia isless: -0.0 before 0.0, all NaNs tie after +Inf."""
    v = np.array([-np.inf, -1.0, -0.0, -0.0, 0.0, 1.0, np.inf, np.nan, np.nan])
    x = np.array([-0.0, 0.0, np.nan, -np.inf, 5.0, -2.0])
    assert oracle.searchsorted(v, x, "first").tolist() == [2, 4, 7, 0, 6, 1]
    assert oracle.searchsorted(v, x, "last").tolist() == [3, 4, 8, 0, 5, 0]
    vd = v[::-1].copy()  # the descending sequence (rev=true)
    assert oracle.searchsorted(vd, x, "first", "descending").tolist() == [5, 4, 0, 8, 3, 8]
    assert oracle.searchsorted(vd, x, "last", "descending").tolist() == [6, 4, 1, 8, 2, 7]
    # negative NaN payloads tie with positive ones
    neg_nan = np.array([0xFFF8000000000001], dtype=np.uint64).view(np.float64)
    assert oracle.searchsorted(v, neg_nan, "first").tolist() == [7]
    assert oracle.searchsorted(v, neg_nan, "last").tolist() == [8]


def test_searchsorted_empty_and_degenerate():
    x = np.array([3, 1, 7], dtype=np.int32)
    empty = np.array([], dtype=np.int32)
    assert oracle.searchsorted(empty, x, "first").tolist() == [0, 0, 0]
    assert oracle.searchsorted(empty, x, "last").tolist() == [-1, -1, -1]
    assert oracle.searchsorted(np.array([1, 3, 5], dtype=np.int32), empty).size == 0
    same = np.full(10, 4, dtype=np.int32)  # all equal: first = 0 or n, last = -1 or n - 1
    q = np.array([3, 4, 5], dtype=np.int32)
    assert oracle.searchsorted(same, q, "first").tolist() == [0, 0, 10]
    assert oracle.searchsorted(same, q, "last").tolist() == [-1, 9, 9]


# ------------------------------------------------------------ accumulate
# Sec. II-B: accumulate (prefix scan), inclusive and exclusive.  Pinned against
# numpy's cumulative routines where they agree with the definition, exact
# rational prefix sums (math.fsum), hand-worked Julia max/min facts, and the
# exclusive = shifted inclusive invariant.

INT_DTYPES = [np.uint16, np.int16, np.uint32, np.int32, np.uint64, np.int64]


@pytest.mark.parametrize("dtype", INT_DTYPES)
def test_accumulate_integers_match_numpy(dtype):
    """Wrapping + and plain max/min on integers are numpy's cumsum (in the
    key's width) and maximum/minimum.accumulate."""
    x = synth.random_keys(3000, dtype, seed=101)
    assert np.array_equal(oracle.accumulate(x, "add"), np.cumsum(x, dtype=dtype))
    assert np.array_equal(oracle.accumulate(x, "max"), np.maximum.accumulate(x))
    assert np.array_equal(oracle.accumulate(x, "min"), np.minimum.accumulate(x))
    # a start value enters every prefix
    init = dtype(7)
    with np.errstate(over="ignore"):
        want = (np.cumsum(x, dtype=dtype) + init).astype(dtype)
    assert np.array_equal(oracle.accumulate(x, "add", init=init), want)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("op", ["add", "max", "min"])
def test_exclusive_is_shifted_inclusive(dtype, op):
    x = synth.random_keys(500, dtype, seed=102, mode="dups")
    if np.dtype(dtype).kind == "f":
        x = x[~np.isnan(x)]
        x = x[np.isfinite(x)] if op == "add" else x
    init = oracle.identity(dtype, op)
    inc = oracle.accumulate(x, op, True, init)
    exc = oracle.accumulate(x, op, False, init)
    assert bits_equal(exc[:1], np.array([init], dtype=dtype))
    assert bits_equal(exc[1:], inc[:-1])


def bits_equal(a, b):
    a, b = np.ascontiguousarray(a), np.ascontiguousarray(b)
    if a.shape != b.shape:
        return False
    u = np.dtype(f"u{a.dtype.itemsize}")
    return bool(np.array_equal(a.view(u), b.view(u)))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_accumulate_float_add_against_exact_prefix_sums(dtype):
    """Each output is the exact prefix sum (math.fsum, correctly rounded in
    float64) rounded to the key's type, to within one float64 rounding before
    that last step: equal for float32, within 2 ulp for float64.  Mixed signs
    and magnitudes make a plain float64 running sum visibly worse."""
    n = 1500
    u = synth.u01_f64(103, n)
    mag = np.exp2(np.floor(synth.u01_f64(104, n) * 40) - 20)
    x = ((u - 0.5) * mag).astype(dtype)
    got = oracle.accumulate(x, "add")
    xs = x.astype(np.float64).tolist()
    exact = np.array([math.fsum(xs[: i + 1]) for i in range(n)])
    if dtype == np.float32:
        assert np.array_equal(got, exact.astype(np.float32))
    else:
        assert np.all(np.abs(got - exact) <= 2 * np.spacing(np.abs(exact)))


def test_accumulate_integer_valued_floats_are_exact():
    """Sums of small integers are exact in any order: numpy's cumsum agrees bit
    for bit, and so does the exclusive form from a start value."""
    x = (synth.splitmix64(105, 4000) % np.uint64(2001)).astype(np.float64) - 1000.0
    assert np.array_equal(oracle.accumulate(x, "add"), np.cumsum(x))
    ex = oracle.accumulate(x.astype(np.float32), "add", inclusive=False, init=np.float32(5))
    assert np.array_equal(ex, np.concatenate([[5.0], 5.0 + np.cumsum(x)[:-1]]).astype(np.float32))


def test_accumulate_julia_max_min_and_specials_by_hand():
    """Julia facts: max(-0.0, 0.0) == 0.0, min(-0.0, 0.0) == -0.0, a NaN operand
    makes max and min NaN; IEEE: Inf + 1 = Inf, Inf + (-Inf) = NaN, and a sum
    of negative zeros stays -0.0."""
    nan, inf = np.nan, np.inf
    got = oracle.accumulate(np.array([-0.0, 0.0, -0.0]), "max", init=-0.0)
    assert bits_equal(got, np.array([-0.0, 0.0, 0.0]))
    got = oracle.accumulate(np.array([0.0, -0.0, 0.0]), "min", init=0.0)
    assert bits_equal(got, np.array([0.0, -0.0, -0.0]))
    got = oracle.accumulate(np.array([1.0, nan, 5.0], np.float32), "max")
    assert got[0] == 1.0 and np.isnan(got[1]) and np.isnan(got[2])
    got = oracle.accumulate(np.array([3.0, 2.0, nan, -9.0]), "min")
    assert got[:2].tolist() == [3.0, 2.0] and np.isnan(got[2:]).all()
    got = oracle.accumulate(np.array([1.0, inf, 2.0, -inf, 3.0]), "add")
    assert got[:3].tolist() == [1.0, inf, inf] and np.isnan(got[3:]).all()
    assert bits_equal(oracle.accumulate(np.array([-0.0, -0.0]), "add", init=-0.0), np.array([-0.0, -0.0]))
    # identities: the lowest / highest value of the type, -Inf / +Inf for floats
    assert oracle.identity(np.int16, "max") == -32768 and oracle.identity(np.uint32, "min") == 2**32 - 1
    assert oracle.identity(np.float64, "max") == -inf and oracle.identity(np.float32, "add") == 0


def test_accumulate_empty_and_single():
    for dtype in DTYPES:
        e = np.array([], dtype=dtype)
        assert oracle.accumulate(e, "add").size == 0
        one = synth.random_keys(1, dtype, seed=106, mode="narrow")
        assert bits_equal(oracle.accumulate(one, "max"), one)
        assert bits_equal(oracle.accumulate(one, "add", inclusive=False, init=dtype(3)), np.array([3], dtype=dtype))


# ------------------------------------------------------------ 16-bit floats
# IEEE binary16 (numpy float16) and bfloat16 (its uint16 bits, as_dtype=
# "bfloat16"), ordered by Julia isless through their exact float32 values.

def _bf16_value(bits):
    """bfloat16 bits -> float32 values: the bits are the top half of a float32."""
    return (np.asarray(bits, dtype=np.uint32) << np.uint32(16)).view(np.float32)


def test_float16_isless_facts_by_hand():
    """Bit patterns read off the binary16 layout (sign | 5-bit exponent |
    10-bit fraction): -0.0 before +0.0; every NaN after +Inf and tied; the
    smallest subnormal above +0.0; 65504 the largest finite value."""
    pairs = [(0x8000, 0x0000, True), (0x0000, 0x8000, False), (0x7C00, 0x7E00, True),
             (0x7E00, 0x7C00, False), (0x7E00, 0xFE01, False), (0xFE01, 0x7E00, False),
             (0x0000, 0x0001, True), (0x7BFF, 0x7C00, True), (0xFC00, 0xFBFF, True),
             (0x3C00, 0x4000, True), (0xBC00, 0x3C00, True), (0x8001, 0x8000, True)]
    a = np.array([p[0] for p in pairs], np.uint16).view(np.float16)
    b = np.array([p[1] for p in pairs], np.uint16).view(np.float16)
    assert oracle.isless(a, b).tolist() == [p[2] for p in pairs]


def test_bfloat16_isless_facts_by_hand():
    """bfloat16 = the top 16 bits of a float32: 0x3F80 is 1.0, 0x7F80 +Inf,
    0x7FC0 a NaN, 0x8000 -0.0, 0x0001 the smallest subnormal."""
    pairs = [(0x8000, 0x0000, True), (0x7F80, 0x7FC0, True), (0xFFC0, 0x7FC0, False),
             (0x3F80, 0x4000, True), (0xBF80, 0x0000, True), (0x0000, 0x0001, True),
             (0x7F7F, 0x7F80, True), (0xFF80, 0xFF7F, True)]
    a = np.array([p[0] for p in pairs], np.uint16)
    b = np.array([p[1] for p in pairs], np.uint16)
    assert oracle.isless(a, b, as_dtype="bfloat16").tolist() == [p[2] for p in pairs]
    assert _bf16_value(np.array([0x3F80]))[0] == 1.0


def test_float16_matches_numpy_comparison():
    """Off NaNs and signed zeros, isless is numpy's float16 <."""
    a = synth.random_keys(20000, np.float16, seed=121)
    b = synth.random_keys(20000, np.float16, seed=122)
    ok = ~np.isnan(a) & ~np.isnan(b) & ~((a == 0) & (b == 0))
    assert np.array_equal(oracle.isless(a[ok], b[ok]), a[ok] < b[ok])


@pytest.mark.parametrize("mode", ["bits", "dups", "narrow"])
@pytest.mark.parametrize("desc", [False, True])
def test_16bit_floats_match_python_timsort(mode, desc):
    h = synth.random_keys(3000, np.float16, seed=123, mode=mode)
    pyvals = [float(v) for v in h]
    want = sorted(range(h.size), key=lambda i: _py_key(pyvals[i]), reverse=desc)
    assert np.array_equal(oracle.sortperm(h, "descending" if desc else "ascending"), np.array(want))
    bits = synth.random_keys(3000, np.uint16, seed=124, mode="bits" if mode == "bits" else "dups")
    vals = [float(v) for v in _bf16_value(bits)]
    want = sorted(range(bits.size), key=lambda i: _py_key(vals[i]), reverse=desc)
    got = oracle.sortperm(bits, "descending" if desc else "ascending", as_dtype="bfloat16")
    assert np.array_equal(got, np.array(want))


def test_16bit_floats_search_brute_force():
    v = oracle.sort(synth.random_keys(300, np.float16, seed=125, mode="dups"))
    x = np.concatenate([synth.special_values(np.float16), synth.random_keys(50, np.float16, seed=126)])
    for side in ("first", "last"):
        got = oracle.searchsorted(v, x, side)
        for i in range(x.size):
            xi = np.full(v.size, x[i], dtype=v.dtype)
            want = np.count_nonzero(oracle.isless(v, xi)) if side == "first" \
                else np.count_nonzero(~oracle.isless(xi, v)) - 1
            assert got[i] == want
    with pytest.raises(RuntimeError):
        oracle.accumulate(v, "add")  # 16-bit float scans are not defined in the oracle


# ------------------------------------------------------------ 128-bit integers
# Int128 / UInt128 keys (the paper's best AcceleratedKernels case, Sec. IV-C),
# 16-byte elements, low word first.

def _i128_keys(n, seed, mode):
    lo = synth.splitmix64(seed, n)
    if mode == "bits":
        hi = synth.splitmix64(seed + 1, n)
    else:  # few distinct high words, many ties on the whole key
        hi = synth.special_values(np.int64)[(synth.splitmix64(seed + 1, n) % np.uint64(8)).astype(np.int64)]
        lo = lo % np.uint64(5)
    return oracle.int128_from_words(lo, hi)


def _py_int(lo, hi, signed):
    v = (int(hi) << 64) | int(lo)
    return v - (1 << 128) if signed and v >> 127 else v


@pytest.mark.parametrize("signed", [True, False])
@pytest.mark.parametrize("mode", ["bits", "dups"])
@pytest.mark.parametrize("desc", [False, True])
def test_int128_matches_python_ints(signed, mode, desc):
    """Python's arbitrary-precision ints and Timsort define the order."""
    k = _i128_keys(4000, 131, mode)
    lo, hi = oracle.int128_words(k)
    vals = [_py_int(a, b, signed) for a, b in zip(lo.tolist(), hi.tolist())]
    want = sorted(range(k.size), key=lambda i: vals[i], reverse=desc)
    got = oracle.sortperm(k, "descending" if desc else "ascending", as_dtype="int128" if signed else "uint128")
    assert np.array_equal(got, np.array(want))


@pytest.mark.parametrize("signed", [True, False])
def test_int128_matches_numpy_lexsort(signed):
    """Ordering by (high word, signed for Int128; then low word unsigned) is
    the 128-bit order; numpy's lexsort is stable."""
    k = _i128_keys(20000, 132, "dups")
    lo, hi = oracle.int128_words(k)
    want = np.lexsort((lo, hi.view(np.int64) if signed else hi))
    assert np.array_equal(oracle.sortperm(k, as_dtype="int128" if signed else "uint128"), want)


def test_int128_search_gather_and_facts():
    """Hand facts: -1 < 0 signed but 2^128 - 1 > 0 unsigned; 2^64 > 2^64 - 1;
    gather moves all 16 bytes; search counts by brute force."""
    k = oracle.int128_from_words([2**64 - 1, 0, 0, 2**64 - 1], [2**64 - 1, 0, 1, 0])  # -1, 0, 2^64, 2^64-1
    assert oracle.isless(k[:1], k[1:2], as_dtype="int128").tolist() == [True]
    assert oracle.isless(k[:1], k[1:2], as_dtype="uint128").tolist() == [False]
    assert oracle.isless(k[3:4], k[2:3], as_dtype="int128").tolist() == [True]
    s = oracle.sort(k, as_dtype="int128")
    assert [_py_int(a, b, True) for a, b in zip(*[w.tolist() for w in oracle.int128_words(s)])] == \
        [-1, 0, 2**64 - 1, 2**64]
    v = oracle.sort(_i128_keys(300, 133, "dups"), as_dtype="int128")
    x = _i128_keys(40, 134, "dups")
    first = oracle.searchsorted(v, x, "first", as_dtype="int128")
    last = oracle.searchsorted(v, x, "last", as_dtype="int128")
    vl, vh = oracle.int128_words(v)
    vv = [_py_int(a, b, True) for a, b in zip(vl.tolist(), vh.tolist())]
    xl, xh = oracle.int128_words(x)
    for i, (a, b) in enumerate(zip(xl.tolist(), xh.tolist())):
        xi = _py_int(a, b, True)
        assert first[i] == sum(e < xi for e in vv) and last[i] == sum(e <= xi for e in vv) - 1
