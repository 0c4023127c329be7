"""Parity of the batched binary search (Sec. II-B, searchsortedfirst /
searchsortedlast) against the CPU oracle, exact, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.uint16, np.int16, np.uint32, np.int32, np.uint64, np.int64, np.float32, np.float64]
TABLE = {2: 8192, 4: 4096, 8: 2048}  # pivot keys the kernel keeps in shared memory


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _search(ak, v, x, side, order):
    tv, u = to_dev(v)
    tx, _ = to_dev(x)
    f = ak.ak_searchsortedfirst if side == "first" else ak.ak_searchsortedlast
    out = f(tv, tx, order, unsigned=u)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _queries(v, dtype, seed, m):
    """Exact hits, random keys of the dtype, the dtype's special values."""
    hits = v[(synth.splitmix64(seed, m // 2) % np.uint64(max(v.size, 1))).astype(np.int64)] if v.size else v[:0]
    rand = synth.random_keys(m - hits.size, dtype, seed + 1, mode="dups")
    return np.concatenate([hits, rand, synth.special_values(dtype)])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("order", ["ascending", "descending"])
@pytest.mark.parametrize("side", ["first", "last"])
def test_parity_all_dtypes(ak, dtype, order, side):
    """100,003 keys (many table stretches, a ragged last one) with duplicates
    and special values; queries: hits, random keys, specials."""
    keys = np.concatenate([synth.random_keys(60_000, dtype, seed=81, mode="dups"),
                           synth.random_keys(40_003 - synth.special_values(dtype).size, dtype, seed=82),
                           synth.special_values(dtype)])
    v = oracle.sort(keys, order)
    x = _queries(v, dtype, 83, 50_001)
    got = _search(ak, v, x, side, order)
    np.testing.assert_array_equal(got, oracle.searchsorted(v, x, side, order))


@pytest.mark.parametrize("dtype", [np.uint16, np.float32, np.float64])
def test_sizes_around_the_table(ak, dtype):
    """n = 0, 1, 2, a few, and the table size -1, +0, +1, +2 (K = n - 1 up to
    the full table), m = 1 and m not a multiple of the block."""
    k = TABLE[np.dtype(dtype).itemsize]
    for n in (0, 1, 2, 3, 31, k - 1, k, k + 1, k + 2, 3 * k + 7):
        v = oracle.sort(synth.random_keys(n, dtype, seed=84 + n, mode="dups"))
        for m in (1, 513):
            x = _queries(v, dtype, 85 + n, m)
            for side in ("first", "last"):
                got = _search(ak, v, x, side, "ascending")
                np.testing.assert_array_equal(got, oracle.searchsorted(v, x, side), err_msg=f"n={n} m={m} {side}")


def test_empty_queries_and_all_equal_keys(ak):
    v = np.full(10_000, 7, dtype=np.int32)
    empty = np.array([], dtype=np.int32)
    assert _search(ak, v, empty, "first", "ascending").size == 0
    x = np.array([6, 7, 8], dtype=np.int32)
    assert _search(ak, v, x, "first", "ascending").tolist() == [0, 0, 10_000]
    assert _search(ak, v, x, "last", "ascending").tolist() == [-1, 9_999, 9_999]
    assert _search(ak, v, x, "first", "descending").tolist() == [10_000, 0, 0]
    assert _search(ak, v, x, "last", "descending").tolist() == [9_999, 9_999, -1]


def test_queries_are_the_keys_themselves(ak):
    """x = v (the same device array): every first/last brackets the run of keys
    equal to each one."""
    v = oracle.sort(synth.random_keys(200_000, np.float32, seed=86, mode="dups"))
    tv, _ = to_dev(v)
    first = ak.ak_searchsortedfirst(tv, tv).cpu().numpy()
    last = ak.ak_searchsortedlast(tv, tv).cpu().numpy()
    np.testing.assert_array_equal(first, oracle.searchsorted(v, v, "first"))
    np.testing.assert_array_equal(last, oracle.searchsorted(v, v, "last"))
    idx = np.arange(v.size)
    assert np.all(first <= idx) and np.all(last >= idx)


def test_out_argument_and_stream(ak):
    v = np.sort(synth.random_keys(50_000, np.int64, seed=87, mode="narrow"))
    x = synth.random_keys(10_000, np.int64, seed=88, mode="narrow")
    tv, tx = torch.from_numpy(v).cuda(), torch.from_numpy(x).cuda()
    out = torch.full((x.size,), -7, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())  # the fill above runs on the default stream
    with torch.cuda.stream(s):
        r = ak.ak_searchsortedlast(tv, tx, out=out, stream=s)
    s.synchronize()
    assert r is out
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.searchsorted(v, x, "last"))
    with pytest.raises(ValueError):
        ak.ak_searchsortedfirst(tv, tx, out=torch.empty(3, dtype=torch.int64, device="cuda"))
    with pytest.raises(TypeError):
        ak.ak_searchsortedfirst(tv, tx.to(torch.int32))


@pytest.mark.slow
def test_full_size_sampled(ak):
    """134,217,728 ascending float64 keys (1 GiB, 25% equal neighbours) and
    16,777,216 queries, in the launch configuration the benchmark times;
    20,000 sampled answers against the oracle, and every answer checked for
    range and monotonicity in the query."""
    n, m = 1 << 27, 1 << 24
    v = synth.ascending_f64(n, seed=40)
    u = synth.u01_f64(89, m) * (v[-1] * 1.0002) - v[-1] * 0.0001
    x = np.concatenate([u[: m // 2], v[(synth.splitmix64(90, m - m // 2) % np.uint64(n)).astype(np.int64)]])
    tv, tx = torch.from_numpy(v).cuda(), torch.from_numpy(x).cuda()
    first = ak.ak_searchsortedfirst(tv, tx).cpu().numpy()
    last = ak.ak_searchsortedlast(tv, tx).cpu().numpy()
    pick = (synth.splitmix64(91, 20_000) % np.uint64(m)).astype(np.int64)
    np.testing.assert_array_equal(first[pick], oracle.searchsorted(v, x[pick], "first"))
    np.testing.assert_array_equal(last[pick], oracle.searchsorted(v, x[pick], "last"))
    assert first.min() >= 0 and first.max() <= n and last.min() >= -1 and last.max() <= n - 1
    assert np.all(last >= first - 1)
    o = np.argsort(x, kind="stable")
    assert np.all(np.diff(first[o]) >= 0) and np.all(np.diff(last[o]) >= 0)


TILE = 4096  # queries per CTA iteration; a tile in v's order takes the shared window


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("order", ["ascending", "descending"])
@pytest.mark.parametrize("side", ["first", "last"])
def test_sorted_query_tiles(ak, dtype, order, side):
    """Queries in v's own order (duplicates, hits, specials): every tile is
    answered through the shared-memory window; three whole tiles and a ragged
    one."""
    keys = np.concatenate([synth.random_keys(60_000, dtype, seed=181, mode="dups"),
                           synth.random_keys(40_003 - synth.special_values(dtype).size, dtype, seed=182),
                           synth.special_values(dtype)])
    v = oracle.sort(keys, order)
    x = oracle.sort(_queries(v, dtype, 183, 3 * TILE + 5 - synth.special_values(dtype).size), order)
    assert x.size == 3 * TILE + 5
    got = _search(ak, v, x, side, order)
    np.testing.assert_array_equal(got, oracle.searchsorted(v, x, side, order))


@pytest.mark.parametrize("dtype", [np.uint16, np.float32, np.int64])
def test_sorted_queries_tile_boundaries_and_windows(ak, dtype):
    """m = one tile -1/+0/+1; dense tiles (the window holds the keys between a
    tile's first and last answer) and sparse ones (queries spread over 2M keys:
    the window is above 64 KB and the tile bisects in global memory between its
    bounds)."""
    v = oracle.sort(synth.random_keys(2_000_003, dtype, seed=184, mode="dups"))
    for m in (TILE - 1, TILE, TILE + 1):
        dense = oracle.sort(v[(synth.splitmix64(185 + m, m) % np.uint64(6_000)).astype(np.int64) + 1_000_000])
        sparse = oracle.sort(_queries(v, dtype, 186 + m, m - synth.special_values(dtype).size))
        for x in (dense, sparse):
            for side in ("first", "last"):
                got = _search(ak, v, x, side, "ascending")
                np.testing.assert_array_equal(got, oracle.searchsorted(v, x, side), err_msg=f"m={m} {side}")


def test_mixed_sorted_and_unsorted_tiles(ak):
    """Tiles in order, out of order, in the reverse order and with one
    descent at a tile's last slot, in one batch: each tile takes its own path
    and every answer matches."""
    v = oracle.sort(synth.random_keys(300_000, np.float64, seed=187, mode="dups"))
    q = _queries(v, np.float64, 188, 4 * TILE - synth.special_values(np.float64).size)
    a = oracle.sort(q[:TILE])
    b = q[TILE: 2 * TILE]
    c = oracle.sort(q[2 * TILE: 3 * TILE])[::-1]
    d = oracle.sort(q[3 * TILE:])
    d[-1], d[-2] = d[-2], d[-1]
    x = np.ascontiguousarray(np.concatenate([a, b, c, d]))
    for side in ("first", "last"):
        for order in ("ascending", "descending"):
            vv = oracle.sort(v, order)
            got = _search(ak, vv, x, side, order)
            np.testing.assert_array_equal(got, oracle.searchsorted(vv, x, side, order), err_msg=f"{side} {order}")


@pytest.mark.slow
def test_full_size_ascending_queries_sampled(ak):
    """The benchmark's ascending shape: 2^24 ascending float64 queries in 2^27
    ascending keys (1 GiB): every tile takes the shared-window path; 20,000
    sampled answers against the oracle, every answer in range and monotone."""
    n, m = 1 << 27, 1 << 24
    v = synth.ascending_f64(n, seed=40)
    x = synth.ascending_f64(m, seed=93)
    x *= v[-1] / x[-1]
    tv, tx = torch.from_numpy(v).cuda(), torch.from_numpy(x).cuda()
    first = ak.ak_searchsortedfirst(tv, tx).cpu().numpy()
    last = ak.ak_searchsortedlast(tv, tx).cpu().numpy()
    pick = (synth.splitmix64(94, 20_000) % np.uint64(m)).astype(np.int64)
    np.testing.assert_array_equal(first[pick], oracle.searchsorted(v, x[pick], "first"))
    np.testing.assert_array_equal(last[pick], oracle.searchsorted(v, x[pick], "last"))
    assert first.min() >= 0 and first.max() <= n and last.min() >= -1 and last.max() <= n - 1
    assert np.all(np.diff(first) >= 0) and np.all(np.diff(last) >= 0)
