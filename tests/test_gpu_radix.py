"""Parity of the onesweep radix path (ak_sort / ak_sortperm / ak_sort_pairs)
against the CPU oracle, bit-exact, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import (assert_bits_equal, check_perm_properties, oracle_perm, to_dev,
                            to_host)

pytestmark = pytest.mark.gpu

DTYPES = [np.uint16, np.int16, np.uint32, np.int32, np.uint64, np.int64, np.float32, np.float64]
# sizes around the tile boundaries of every tile configuration plus ragged tails
SIZES = [1, 2, 31, 33, 1000, 1535, 1536, 2048, 2560, 3839, 3840, 3841, 4096, 6144, 7681, 100003]


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _run_sort(ak, keys, desc, options=None):
    t, u = to_dev(keys)
    ak.ak_sort(t, "descending" if desc else "ascending", options=options, unsigned=u)
    torch.cuda.synchronize()
    return to_host(t, keys.dtype)


def _run_perm(ak, keys, desc, options=None):
    t, u = to_dev(keys)
    p = ak.ak_sortperm(t, "descending" if desc else "ascending", options=options, unsigned=u)
    torch.cuda.synchronize()
    assert_bits_equal(to_host(t, keys.dtype), keys, "sortperm modified keys")
    return to_host(p, np.uint32)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("desc", [False, True])
@pytest.mark.parametrize("mode", ["bits", "dups", "narrow"])
def test_sort_matches_oracle(ak, dtype, desc, mode):
    for n in (SIZES if mode == "bits" else [3841, 100003]):
        keys = synth.random_keys(n, dtype, seed=1000 + n, mode=mode)
        want = oracle.gather(keys, oracle_perm(keys, desc))
        assert_bits_equal(_run_sort(ak, keys, desc, {"path": ak.AK_PATH_RADIX}), want, f"sort n={n}")


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("desc", [False, True])
@pytest.mark.parametrize("mode", ["bits", "dups"])
def test_sortperm_matches_oracle(ak, dtype, desc, mode):
    for n in ([1, 3840, 3841, 100003] if mode == "bits" else [5000, 100003]):
        keys = synth.random_keys(n, dtype, seed=2000 + n, mode=mode)
        want = oracle_perm(keys, desc).astype(np.uint32)
        assert np.array_equal(_run_perm(ak, keys, desc, {"path": ak.AK_PATH_RADIX}), want), f"sortperm n={n}"


@pytest.mark.parametrize("dtype", [np.uint32, np.float64, np.int16, np.float32])
@pytest.mark.parametrize("vdtype", [np.uint8, np.uint16, np.uint32, np.uint64])
@pytest.mark.parametrize("desc", [False, True])
def test_pairs_match_oracle(ak, dtype, vdtype, desc):
    n = 50001
    keys = synth.random_keys(n, dtype, seed=3000, mode="dups")
    vals = synth.splitmix64(3001, n).astype(vdtype)
    p = oracle_perm(keys, desc)
    kt, ku = to_dev(keys)
    vt, _ = to_dev(vals)
    ak.ak_sort_pairs(kt, vt, "descending" if desc else "ascending", options={"path": ak.AK_PATH_RADIX}, unsigned=ku)
    torch.cuda.synchronize()
    assert_bits_equal(to_host(kt, keys.dtype), oracle.gather(keys, p), "pair keys")
    assert_bits_equal(to_host(vt, vals.dtype), oracle.gather(vals, p), "pair values")


def _default_tile(kb, vb):
    """Keys per tile of the default configuration: 512 threads, about 40 KB of
    keys+values per tile, 2..12 keys per thread."""
    return 512 * min(max(40960 // (512 * (kb + vb)), 2), 12)


@pytest.mark.parametrize("dtype", [np.uint16, np.int32, np.float32, np.int64, np.float64])
@pytest.mark.parametrize("vdtype", [None, np.uint8, np.uint32, np.uint64])
def test_default_config_tile_boundaries(ak, dtype, vdtype):
    """The default configuration (40 KB tiles): sort, sortperm and pairs at one
    tile -1/0/+1 and many tiles with a ragged tail, both orders, on keys with
    long runs of equal digits."""
    kb = np.dtype(dtype).itemsize
    vb = 0 if vdtype is None else np.dtype(vdtype).itemsize
    tile = _default_tile(kb, vb if vdtype is not None else 0)
    ptile = _default_tile(kb, 4)  # sortperm carries u32 indices
    rad = {"path": ak.AK_PATH_RADIX}
    for n in sorted({tile - 1, tile, tile + 1, ptile - 1, ptile + 1, 37 * tile + 11}):
        keys = synth.random_keys(n, dtype, seed=7300 + n + kb, mode="dups" if n % 2 else "bits")
        for desc in (False, True):
            order = "descending" if desc else "ascending"
            p = oracle_perm(keys, desc)
            if vdtype is None:
                assert_bits_equal(_run_sort(ak, keys, desc, rad), oracle.gather(keys, p), f"sort n={n}")
                assert np.array_equal(_run_perm(ak, keys, desc, rad), p.astype(np.uint32)), f"sortperm n={n}"
            else:
                vals = synth.splitmix64(7301, n).astype(vdtype)
                kt, ku = to_dev(keys)
                vt, _ = to_dev(vals)
                ak.ak_sort_pairs(kt, vt, order, options=rad, unsigned=ku)
                torch.cuda.synchronize()
                assert_bits_equal(to_host(kt, keys.dtype), oracle.gather(keys, p), f"pair keys n={n}")
                assert_bits_equal(to_host(vt, vals.dtype), oracle.gather(vals, p), f"pair values n={n}")


@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dtype", [np.uint32, np.int64, np.float32, np.uint16])
def test_every_tile_config(ak, cfg, dtype):
    opts = {"tile_config": cfg, "path": ak.AK_PATH_RADIX}
    for n in (1, 1536, 6145, 200001):
        keys = synth.random_keys(n, dtype, seed=4000 + n, mode="dups")
        for desc in (False, True):
            p = oracle_perm(keys, desc)
            assert_bits_equal(_run_sort(ak, keys, desc, opts), oracle.gather(keys, p), f"cfg {cfg} n={n}")
            assert np.array_equal(_run_perm(ak, keys, desc, opts), p.astype(np.uint32))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("vdtype", [None, np.uint8, np.uint16, np.uint32, np.uint64])
def test_lookback_warp_config_tile_boundaries(ak, dtype, vdtype):
    """Tile configuration 4 (the look-back warp): sort, sortperm and pairs of
    every value width, both orders, at one tile -1/0/+1 and several tiles with
    a ragged tail, on heavy-duplicate keys (long runs of equal digits)."""
    opts = {"tile_config": 4, "path": ak.AK_PATH_RADIX}
    kb = np.dtype(dtype).itemsize
    vb = 0 if vdtype is None else np.dtype(vdtype).itemsize
    regs = (kb + 3) // 4 + (vb + 3) // 4 + 1
    items = min(21 // regs, 12)
    if vb == 0 and kb <= 4:
        items = min(items, 8)
    tile = 480 * items  # smem never limits these widths below the register bound
    for n in (tile - 1, tile, tile + 1, 7 * tile + 13):
        keys = synth.random_keys(n, dtype, seed=7000 + n + kb, mode="dups" if n % 2 else "bits")
        for desc in (False, True):
            order = "descending" if desc else "ascending"
            p = oracle_perm(keys, desc)
            if vdtype is None:
                assert_bits_equal(_run_sort(ak, keys, desc, opts), oracle.gather(keys, p), f"ws sort n={n}")
                assert np.array_equal(_run_perm(ak, keys, desc, opts), p.astype(np.uint32)), f"ws sortperm n={n}"
            else:
                vals = synth.splitmix64(7001, n).astype(vdtype)
                kt, ku = to_dev(keys)
                vt, _ = to_dev(vals)
                ak.ak_sort_pairs(kt, vt, order, options=opts, unsigned=ku)
                torch.cuda.synchronize()
                assert_bits_equal(to_host(kt, keys.dtype), oracle.gather(keys, p), f"ws pair keys n={n}")
                assert_bits_equal(to_host(vt, vals.dtype), oracle.gather(vals, p), f"ws pair values n={n}")


@pytest.mark.parametrize("dtype", [np.uint32, np.int64, np.float32, np.float64])
def test_lookback_warp_config_many_tiles_per_cta(ak, dtype):
    """Tile configuration 4 with several tiles per persistent CTA (5M keys:
    every CTA rotates through its three tile buffers and both look-back slots
    more than once); sort, sortperm and pairs against the oracle."""
    opts = {"tile_config": 4, "path": ak.AK_PATH_RADIX}
    n = 5_000_003
    keys = synth.random_keys(n, dtype, seed=7100, mode="bits")
    p = oracle_perm(keys, False, threads=8)
    assert_bits_equal(_run_sort(ak, keys, False, opts), oracle.gather(keys, p), "ws sort, many tiles")
    assert np.array_equal(_run_perm(ak, keys, False, opts), p.astype(np.uint32)), "ws sortperm, many tiles"
    vals = np.arange(n, dtype=np.uint32)
    kt, ku = to_dev(keys)
    vt, _ = to_dev(vals)
    ak.ak_sort_pairs(kt, vt, options=opts, unsigned=ku)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(vt, np.uint32), p.astype(np.uint32)), "ws pairs, many tiles"


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("vdtype", [None, np.uint8, np.uint16, np.uint32, np.uint64])
def test_reduce_then_scan_config_tile_boundaries(ak, dtype, vdtype):
    """Tile configuration 5 (upsweep counts per chunk, then chunk-ordered
    passes without look-back): sort, sortperm and pairs of every value width,
    both orders, one tile -1/0/+1, several tiles with a ragged tail, on heavy
    duplicates and on all bit patterns."""
    opts = {"tile_config": 5, "path": ak.AK_PATH_RADIX}
    kb = np.dtype(dtype).itemsize
    vb = 0 if vdtype is None else np.dtype(vdtype).itemsize
    tile = _default_tile(kb, vb)
    ptile = _default_tile(kb, 4)  # sortperm carries u32 indices
    sizes = {tile - 1, tile, tile + 1, 37 * tile + 11} | ({ptile - 1, ptile + 1} if vdtype is None else set())
    for n in sorted(sizes):
        keys = synth.random_keys(n, dtype, seed=7500 + n + kb, mode="dups" if n % 2 else "bits")
        for desc in (False, True):
            order = "descending" if desc else "ascending"
            p = oracle_perm(keys, desc)
            if vdtype is None:
                assert_bits_equal(_run_sort(ak, keys, desc, opts), oracle.gather(keys, p), f"rts sort n={n}")
                assert np.array_equal(_run_perm(ak, keys, desc, opts), p.astype(np.uint32)), f"rts sortperm n={n}"
            else:
                vals = synth.splitmix64(7501, n).astype(vdtype)
                kt, ku = to_dev(keys)
                vt, _ = to_dev(vals)
                ak.ak_sort_pairs(kt, vt, order, options=opts, unsigned=ku)
                torch.cuda.synchronize()
                assert_bits_equal(to_host(kt, keys.dtype), oracle.gather(keys, p), f"rts pair keys n={n}")
                assert_bits_equal(to_host(vt, vals.dtype), oracle.gather(vals, p), f"rts pair values n={n}")


@pytest.mark.parametrize("dtype", [np.uint32, np.int64, np.float32, np.float64, np.uint16])
def test_reduce_then_scan_config_many_tiles_per_chunk(ak, dtype):
    """Tile configuration 5 where every chunk holds several tiles (5M keys: a
    CTA carries its running digit offsets across tiles, chunks fewer than a
    wave after rounding) and where the key pointer is off 16-byte alignment
    (the upsweep and the pass fall back to plain loads)."""
    opts = {"tile_config": 5, "path": ak.AK_PATH_RADIX}
    n = 5_000_003
    keys = synth.random_keys(n, dtype, seed=7600, mode="bits")
    for desc in (False, True):
        p = oracle_perm(keys, desc, threads=8)
        assert_bits_equal(_run_sort(ak, keys, desc, opts), oracle.gather(keys, p), "rts sort, many tiles")
        assert np.array_equal(_run_perm(ak, keys, desc, opts), p.astype(np.uint32)), "rts sortperm, many tiles"
    vals = np.arange(n, dtype=np.uint32)
    p = oracle_perm(keys, False, threads=8)
    kt, ku = to_dev(keys)
    vt, _ = to_dev(vals)
    ak.ak_sort_pairs(kt, vt, options=opts, unsigned=ku)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(vt, np.uint32), p.astype(np.uint32)), "rts pairs, many tiles"
    base = synth.random_keys(2_000_001, dtype, seed=7601, mode="dups")
    t, u = to_dev(base)
    sub = t[1:]
    ak.ak_sort(sub, options=opts, unsigned=u)
    torch.cuda.synchronize()
    assert_bits_equal(to_host(sub, base.dtype), oracle.gather(base[1:], oracle_perm(base[1:], False, threads=8)),
                      "rts unaligned")
    assert_bits_equal(to_host(t, base.dtype)[:1], base[:1], "rts unaligned: the element before is untouched")


def _packed_patterns(n, dtype, seed):
    """8-byte keys whose active digit passes fall in every arrangement the
    packed sortperm plans for: all passes; only the upper half (the first
    upper pass packs); one upper pass alone (no packing); one lower and one
    upper pass; only the lower half (no upper pass); special values."""
    r = synth.splitmix64(seed, n)
    u = np.dtype(dtype)
    bits = {
        "all": r,
        # floats: positive and finite, so the radix key's lower half stays zero
        "upper_only": r & np.uint64(0x3FFFFFFF00000000 if u.kind == "f" else 0xFFFFFFFF00000000),
        "one_upper": (r & np.uint64(0x0000FF0000000000)) | np.uint64(0x4010000000000000),
        "one_lower_one_upper": (r & np.uint64(0x00FF0000000000FF)) | np.uint64(0x3FF0000000000000),
        "lower_only": (r & np.uint64(0x00000000FFFFFFFF)) | np.uint64(0x4000000000000000),
        "dups": r % np.uint64(7) << np.uint64(37),
    }
    out = {k: v.view(u) for k, v in bits.items()}
    if u.kind == "f":
        out["specials"] = np.resize(synth.special_values(dtype), n)
    return out


@pytest.mark.parametrize("dtype", [np.int64, np.uint64, np.float64])
@pytest.mark.parametrize("desc", [False, True])
def test_sortperm_packed_upper_passes(ak, dtype, desc):
    """ak_sortperm of 8-byte keys packs (upper radix-key half, index) into one
    word for the passes of the upper half: the permutation equals the oracle's
    for every arrangement of active passes, across both tile shapes (3,072
    keys with an index, 5,120 packed words), and equals the unpacked run
    (AK_DEBUG_NO_PACK)."""
    rad = {"path": ak.AK_PATH_RADIX}
    nopack = {"path": ak.AK_PATH_RADIX, "debug_flags": ak.AK_DEBUG_NO_PACK}
    for n in (1, 2, 3071, 3073, 5119, 5121, 200_003):
        for name, keys in _packed_patterns(n, dtype, seed=8800 + n).items():
            want = oracle_perm(keys, desc).astype(np.uint32)
            got = _run_perm(ak, keys, desc, rad)
            assert np.array_equal(got, want), (name, n)
            if n == 200_003:
                assert np.array_equal(_run_perm(ak, keys, desc, nopack), want), (name, n, "no pack")


@pytest.mark.parametrize("dtype", [np.int64, np.float64])
def test_sortperm_packed_many_tiles_per_cta(ak, dtype):
    """Packed sortperm with several tiles per persistent CTA in both tile
    shapes (5M keys), all passes active and upper half only, and the info
    block's pass count."""
    n = 5_000_003
    pats = _packed_patterns(n, dtype, seed=8900)
    for name in ("all", "upper_only"):
        keys = pats[name]
        want = oracle_perm(keys, False, threads=8).astype(np.uint32)
        t, u = to_dev(keys)
        rad = {"path": ak.AK_PATH_RADIX}
        temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORTPERM, n, ak.AK_I64, options=rad), t.device)
        p = ak.ak_sortperm(t, temp=temp, options=rad, unsigned=u)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(p, np.uint32), want), name
        assert ak.ak_status_check(temp) == 0
        assert ak.ak_last_info(temp)["radix_passes"] == (8 if name == "all" else 4)


def test_trivial_passes_and_all_equal(ak):
    # every key equal: all passes trivial; sortperm must be the identity
    keys = np.full(70000, 7, dtype=np.int64)
    assert np.array_equal(_run_perm(ak, keys, False), np.arange(70000, dtype=np.uint32))
    assert np.array_equal(_run_perm(ak, keys, True), np.arange(70000, dtype=np.uint32))
    # NaNs only, different payloads: input order must survive
    nan = (np.uint32(0x7FC00000) | (np.arange(5000, dtype=np.uint32) * 7919 % 4093)).view(np.float32)
    assert_bits_equal(_run_sort(ak, nan, False), nan, "all-NaN sort")
    # an odd number of moving passes (copy-back): only byte 1 varies
    k = (synth.splitmix64(5, 30000) % np.uint64(256)).astype(np.uint32) << np.uint32(8)
    k |= np.uint32(0x11000000)
    info_keys, u = to_dev(k)
    rad = {"path": ak.AK_PATH_RADIX}
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, k.size, ak.AK_U32, options=rad), info_keys.device)
    ak.ak_sort(info_keys, temp=temp, options=rad, unsigned=u)
    info = ak.ak_last_info(temp)
    assert info["radix_passes"] == 1 and info["status"] == 0
    assert_bits_equal(to_host(info_keys, k.dtype), np.sort(k), "copy-back")


def test_special_values_every_dtype(ak):
    for dt in DTYPES:
        sv = synth.special_values(dt)
        keys = np.tile(sv, 300)[: 4000]
        for desc in (False, True):
            p = oracle_perm(keys, desc)
            assert_bits_equal(_run_sort(ak, keys, desc), oracle.gather(keys, p), f"{dt}")


def test_unaligned_pointers_take_plain_loads(ak):
    # key pointer offset by one element: no 16-byte alignment, still exact
    base = synth.random_keys(100001, np.uint32, seed=77, mode="bits")
    t, _ = to_dev(base)
    sub = t[1:]
    ak.ak_sort(sub, options={"path": ak.AK_PATH_RADIX}, unsigned=True)
    torch.cuda.synchronize()
    want = oracle.sort(base[1:])
    assert_bits_equal(to_host(sub, np.uint32), want, "unaligned")
    assert to_host(t, np.uint32)[0] == base[0]


def test_empty_and_errors(ak):
    t = torch.empty(0, dtype=torch.float32, device="cuda")
    ak.ak_sort(t)
    assert ak.ak_sortperm(t).numel() == 0
    with pytest.raises(ak.AkError):
        ak.ak_sort(torch.zeros(10, device="cuda"), temp=torch.empty(16, dtype=torch.uint8, device="cuda"))


@pytest.mark.parametrize("cfg", [0, 4])
def test_lookback_timeout_reports_status(ak, cfg):
    """The test hook leaves tile 0 of every pass unowned: tile 1's look-back
    must give up after timeout_ns and the status word must say so."""
    keys = synth.random_keys(20000, np.uint32, seed=9, mode="bits")
    t, u = to_dev(keys)
    opts = {"path": ak.AK_PATH_RADIX, "timeout_ns": 2_000_000, "debug_flags": ak.AK_DEBUG_SKIP_FIRST_TILE,
            "tile_config": cfg}
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, keys.size, ak.AK_U32, options=opts), t.device)
    ak.ak_sort(t, temp=temp, options=opts, unsigned=u)
    assert ak.ak_status_check(temp) == 5
    # the context is still usable and a normal call clears the status (the
    # failed call left unspecified keys behind, so restore them first)
    t.copy_(to_dev(keys)[0])
    ak.ak_sort(t, temp=temp, options={"path": ak.AK_PATH_RADIX}, unsigned=u)
    assert ak.ak_status_check(temp) == 0
    assert_bits_equal(to_host(t, np.uint32), np.sort(keys), "after timeout")


def test_stream_and_graph_capture(ak):
    keys = synth.random_keys(300000, np.float32, seed=12, mode="bits")
    t, _ = to_dev(keys)
    pristine = t.clone()
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, keys.size, ak.AK_F32), t.device)
    s = torch.cuda.Stream()
    ak.ak_sort(t, temp=temp, stream=s)  # warm up (sets kernel attributes outside capture)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ak.ak_sort(t, temp=temp, stream=s)
    for _ in range(3):
        t.copy_(pristine)
        g.replay()
    torch.cuda.synchronize()
    assert_bits_equal(to_host(t, np.float32), oracle.sort(keys), "graph replay")


@pytest.mark.slow
@pytest.mark.parametrize("which", ["i64", "f32"])
def test_full_size_268M(ak, which):
    """268,435,456 keys: int64 uniform over all bit patterns and float32 N(0,1)
    with 0.1% NaN and 0.1% -0.0; sortperm verified by the stable-sortperm
    properties, then sort compared bit-exactly with keys[perm]."""
    n = 268_435_456
    RADIX = {"path": ak.AK_PATH_RADIX}
    keys = synth.uniform_i64(n, seed=2) if which == "i64" else synth.normal_f32_special(n, seed=3)
    for desc in (False,):
        t, u = to_dev(keys)
        p = ak.ak_sortperm(t, "descending" if desc else "ascending", options=RADIX, unsigned=u)
        torch.cuda.synchronize()
        perm = to_host(p, np.uint32)
        del p
        check_perm_properties(keys, perm, desc)
        ak.ak_sort(t, "descending" if desc else "ascending", options=RADIX, unsigned=u)
        torch.cuda.synchronize()
        assert_bits_equal(to_host(t, keys.dtype), keys[perm.astype(np.int64)], "full-size sort")
        del t
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("desc", [False, True])
def test_sortperm_lowmem_matches_oracle(ak, dtype, desc):
    """ak_sortperm_lowmem (Sec. II-B sortperm_lowmem): the permutation of
    ak_sortperm from a workspace without key copies, keys read through the
    index in every pass."""
    for n in (1, 2, 3841, 6145, 100_003):
        keys = synth.random_keys(n, dtype, seed=9000 + n, mode="dups" if n % 2 else "bits")
        want = oracle_perm(keys, desc).astype(np.uint32)
        t, u = to_dev(keys)
        p = ak.ak_sortperm_lowmem(t, "descending" if desc else "ascending", unsigned=u)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(p, np.uint32), want), (np.dtype(dtype), n, desc)
        assert_bits_equal(to_host(t, keys.dtype), keys, "lowmem keeps the keys")


def test_sortperm_lowmem_configs_unaligned_and_many_tiles(ak):
    keys = synth.random_keys(3_000_001, np.float64, seed=9100, mode="bits")
    want = oracle_perm(keys, False, threads=8).astype(np.uint32)
    for cfg in (0, 1, 2, 3, 4, 5):
        t, _ = to_dev(keys)
        p = ak.ak_sortperm_lowmem(t, options={"tile_config": cfg})
        torch.cuda.synchronize()
        assert np.array_equal(to_host(p, np.uint32), want), cfg
    base = synth.random_keys(200_001, np.int32, seed=9101, mode="bits")
    t, _ = to_dev(base)
    p = ak.ak_sortperm_lowmem(t[1:])  # keys off 16-byte alignment
    torch.cuda.synchronize()
    assert np.array_equal(to_host(p, np.uint32), oracle_perm(base[1:], False).astype(np.uint32))

