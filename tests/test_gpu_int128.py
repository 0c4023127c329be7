"""128-bit integer keys (Int128 / UInt128, the widest type of the paper's
local-sort benchmarks) through the radix path and the binary search, bit-exact
against the oracle: sort, sortperm, sortperm_lowmem and key-value sorts of
every value width, both orders, around the 2,048-key tile and across many
tiles; sorted and unsorted query tiles."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TILE = 2048  # keys per tile of the digit pass for 16-byte keys (512 threads x 4)


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _keys(n, seed, mode):
    """V16 keys: all bit patterns, or few distinct high words and many ties,
    or the extremes (0, -1, the smallest and largest signed values)."""
    lo = synth.splitmix64(seed, n)
    if mode == "bits":
        hi = synth.splitmix64(seed + 1, n)
    elif mode == "dups":
        hi = synth.special_values(np.int64)[(synth.splitmix64(seed + 1, n) % np.uint64(8)).astype(np.int64)]
        lo = lo % np.uint64(5)
    else:  # extremes
        pick = (synth.splitmix64(seed + 1, n) % np.uint64(4)).astype(np.int64)
        lo = np.array([0, 2**64 - 1, 0, 2**64 - 1], dtype=np.uint64)[pick]
        hi = np.array([0, 2**64 - 1, 2**63, 2**63 - 1], dtype=np.uint64)[pick]
    return oracle.int128_from_words(lo, hi)


def _dev(k):
    return torch.from_numpy(np.ascontiguousarray(k).view(np.int64).reshape(-1, 2).copy()).cuda()


def _host(t):
    return t.cpu().numpy().reshape(-1).view(np.dtype("V16"))


def _bits(k):
    return np.ascontiguousarray(k).view(np.uint64)


@pytest.mark.parametrize("signed", [True, False])
@pytest.mark.parametrize("mode", ["bits", "dups", "extremes"])
def test_sort_sortperm_lowmem(ak, signed, mode):
    as_dtype = "int128" if signed else "uint128"
    for n in (1, TILE - 1, TILE, TILE + 1, 7 * TILE + 13, 300_007):
        k = _keys(n, 9000 + n, mode)
        for desc in (False, True):
            order = "descending" if desc else "ascending"
            p = oracle.sortperm(k, order, as_dtype=as_dtype)
            t = _dev(k)
            ak.ak_sort(t, order, unsigned=not signed, wide=True)
            torch.cuda.synchronize()
            assert np.array_equal(_bits(_host(t)), _bits(k[p])), (n, mode, desc, "sort")
            t = _dev(k)
            perm = ak.ak_sortperm(t, order, unsigned=not signed, wide=True).cpu().numpy().view(np.uint32)
            assert np.array_equal(perm, p.astype(np.uint32)), (n, mode, desc, "sortperm")
            perm = ak.ak_sortperm_lowmem(t, order, unsigned=not signed, wide=True).cpu().numpy().view(np.uint32)
            assert np.array_equal(perm, p.astype(np.uint32)), (n, mode, desc, "sortperm_lowmem")


@pytest.mark.parametrize("vdtype", [np.uint8, np.uint16, np.uint32, np.uint64])
def test_pairs_every_value_width(ak, vdtype):
    for n in (TILE + 1, 100_003):
        k = _keys(n, 9100 + n, "dups")
        vals = synth.splitmix64(9101, n).astype(vdtype)
        for desc in (False, True):
            order = "descending" if desc else "ascending"
            p = oracle.sortperm(k, order, as_dtype="int128")
            t, v = _dev(k), torch.from_numpy(vals.view(np.dtype(f"i{vals.itemsize}"))).cuda()
            ak.ak_sort_pairs(t, v, order, wide=True)
            torch.cuda.synchronize()
            assert np.array_equal(_bits(_host(t)), _bits(k[p])), (n, desc, "pair keys")
            assert np.array_equal(v.cpu().numpy().view(vdtype), vals[p]), (n, desc, "pair values")


def test_many_tiles_per_cta(ak):
    """4M keys: every persistent CTA walks several tiles in each of the 16 passes."""
    n = 4_000_037
    k = _keys(n, 9200, "bits")
    p = oracle.sortperm(k, threads=8, as_dtype="int128")
    t = _dev(k)
    ak.ak_sort(t, wide=True)
    torch.cuda.synchronize()
    assert np.array_equal(_bits(_host(t)), _bits(k[p]))


@pytest.mark.parametrize("signed", [True, False])
@pytest.mark.parametrize("order", ["ascending", "descending"])
def test_searchsorted(ak, signed, order):
    as_dtype = "int128" if signed else "uint128"
    v = oracle.sort(_keys(50_001, 9300, "dups"), order, as_dtype=as_dtype)
    q = np.concatenate([_keys(3 * 4096, 9301, "dups"), v[::13], _keys(64, 9302, "extremes")])
    for x in (q, oracle.sort(q, order, as_dtype=as_dtype)):  # unsorted, then sorted query tiles
        for side, fn in (("first", ak.ak_searchsortedfirst), ("last", ak.ak_searchsortedlast)):
            want = oracle.searchsorted(v, x, side, order, as_dtype=as_dtype)
            got = fn(_dev(v), _dev(x), order, unsigned=not signed, wide=True).cpu().numpy()
            assert np.array_equal(got, want), (side, signed, order)


def test_refused_operations(ak):
    t = _dev(_keys(100, 9400, "bits"))
    with pytest.raises(ak.AkError) as e:
        ak.ak_sort(t, options={"path": ak.AK_PATH_LEARNED}, wide=True)
    assert e.value.status == 2
    off = torch.tensor([0, 50, 100], dtype=torch.int64, device="cuda")
    lib = ak.load()
    rc = lib.ak_sort_segmented(t.data_ptr(), off.data_ptr(), 2, 100, ak.AK_I128, 0, None, 0, None, None)
    assert rc == 2
    x = torch.zeros((10, 2), dtype=torch.int64, device="cuda")
    assert lib.ak_accumulate(x.data_ptr(), x.data_ptr(), 10, ak.AK_I128, 0, 1, None, None, 0, None, None) == 2


@pytest.mark.slow
def test_int128_large_properties(ak):
    """2^26 signed 128-bit keys (1 GiB) over all bit patterns: the sorted keys
    are in order and the same multiset; the sortperm is a permutation listing
    them in order with ties (none expected) by index; keys[perm] == sorted."""
    n = 1 << 26
    lo, hi = synth.splitmix64(9500, n), synth.splitmix64(9501, n)
    k = oracle.int128_from_words(lo, hi)
    t = _dev(k)
    perm = ak.ak_sortperm(t, wide=True).cpu().numpy().view(np.uint32).astype(np.int64)
    ak.ak_sort(t, wide=True)
    s = t.cpu().numpy().view(np.uint64)
    sl, sh = s[:, 0], s[:, 1].view(np.int64)
    assert np.all((sh[1:] > sh[:-1]) | ((sh[1:] == sh[:-1]) & (sl[1:] >= sl[:-1])))
    assert np.array_equal(np.bincount(perm, minlength=n), np.ones(n, dtype=np.int64))
    assert np.array_equal(sl, lo[perm]) and np.array_equal(s[:, 1], hi[perm])
