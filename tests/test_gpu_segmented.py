"""Parity of the segmented persistent sort and the one-launch block path against
the CPU oracle (bit-exact), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_bits_equal, oracle_perm, to_dev, to_host

pytestmark = pytest.mark.gpu

DTYPES = [np.uint16, np.int16, np.uint32, np.int32, np.uint64, np.int64, np.float32, np.float64]


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _seg_sort(ak, keys, off, desc, graph=False):
    t, u = to_dev(keys)
    o = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int64)).cuda()
    ak.ak_sort_segmented(t, o, "descending" if desc else "ascending", unsigned=u)
    torch.cuda.synchronize()
    return to_host(t, keys.dtype)


def _want(keys, off, desc):
    return oracle.gather(keys, oracle.sortperm_segmented(keys, off, "descending" if desc else "ascending"))


def _mixed_offsets(seed, cap=6144):
    """Empty, single-key, small, at-capacity (cap - 1, cap, cap + 1),
    above-capacity and very large segments."""
    lens = [0, 1, 2, 0, 31, 33, 500, 2047, 2049, cap - 1, cap, cap + 1, 2 * cap + 1, 40000, 3, 0, 70001, 1]
    lens += list(np.diff(synth.lognormal_segments(300, seed=seed, median=300.0, max_len=50000)))
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("desc", [False, True])
@pytest.mark.parametrize("mode", ["bits", "dups"])
def test_segmented_matches_oracle(ak, dtype, desc, mode):
    off = _mixed_offsets(40, ak.ak_segment_capacity(np.dtype(dtype).itemsize))
    keys = synth.random_keys(int(off[-1]), dtype, seed=41, mode=mode)
    assert_bits_equal(_seg_sort(ak, keys, off, desc), _want(keys, off, desc), f"{np.dtype(dtype)}")


def test_bucket_still_above_capacity(ak):
    """A 60,000-key segment whose varying bits are 0-7 and 24: the top-digit
    split leaves two buckets of ~30,000 keys, sorted by global chunked passes."""
    n = 60000
    r = synth.splitmix64(50, n)
    keys = ((r & np.uint64(0xFF)) | ((r >> np.uint64(40)) & np.uint64(1)) << np.uint64(24)).astype(np.uint32)
    off = np.array([0, n], dtype=np.int64)
    for desc in (False, True):
        assert_bits_equal(_seg_sort(ak, keys, off, desc), _want(keys, off, desc), "wide bucket")


def test_segments_all_equal_and_nan_payloads(ak):
    lens = [5000, 9000, 1, 20000]
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    keys = np.empty(int(off[-1]), dtype=np.float32)
    keys[:5000] = 3.0
    nanbits = np.uint32(0x7FC00000) | (np.arange(9000, dtype=np.uint32) % 977)
    keys[5000:14000] = nanbits.view(np.float32)
    keys[14000:14001] = -0.0
    keys[14001:] = synth.normal_f32_special(20000, seed=5, frac=0.05)
    for desc in (False, True):
        assert_bits_equal(_seg_sort(ak, keys, off, desc), _want(keys, off, desc), "special")


def test_lognormal_batch_c4_shape(ak):
    """65,536 segments with lognormal lengths (median 2,048) at 1/16 of the
    batch size: same length distribution shape, uniform u32 keys."""
    off = synth.lognormal_segments(65536 // 16, seed=20, median=2048.0, max_len=1 << 20)
    keys = synth.uniform_u32(int(off[-1]), seed=21)
    assert_bits_equal(_seg_sort(ak, keys, off, False), _want(keys, off, False), "c4 shape")


def test_segmented_graph_replay(ak):
    off = _mixed_offsets(42)
    keys = synth.random_keys(int(off[-1]), np.float64, seed=43, mode="bits")
    t, _ = to_dev(keys)
    pristine = t.clone()
    o = torch.from_numpy(off).cuda()
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT_SEGMENTED, keys.size, ak.AK_F64, nseg=off.size - 1), t.device)
    s = torch.cuda.Stream()
    ak.ak_sort_segmented(t, o, temp=temp, stream=s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ak.ak_sort_segmented(t, o, temp=temp, stream=s)
    for _ in range(2):
        t.copy_(pristine)
        g.replay()
    torch.cuda.synchronize()
    assert_bits_equal(to_host(t, np.float64), _want(keys, off, False), "graph")


def test_segmented_degenerate_inputs(ak):
    t = torch.zeros(0, dtype=torch.int32, device="cuda")
    ak.ak_sort_segmented(t, torch.zeros(1, dtype=torch.int64, device="cuda"))
    keys = synth.random_keys(1000, np.int32, seed=3)
    assert_bits_equal(_seg_sort(ak, keys, np.array([0, 1000]), False), oracle.sort(keys), "one segment")
    assert_bits_equal(_seg_sort(ak, keys, np.arange(0, 1001), False), keys, "all singletons")


@pytest.mark.parametrize("dtype", [np.uint32, np.float64, np.int16])
@pytest.mark.parametrize("n", [1, 2, 100, 2048, 3000, "cap-1", "cap", "cap+1", 100003])
def test_block_path_sort_perm_pairs(ak, dtype, n):
    """AK_PATH_BLOCK: one launch sorts the whole array as a single segment
    (shared memory up to the capacity, MSD split above it).  cap: the
    key-value (8-byte values) capacity, so sort and sortperm sit below theirs."""
    if isinstance(n, str):
        n = ak.ak_segment_capacity(np.dtype(dtype).itemsize, 8) + {"cap-1": -1, "cap": 0, "cap+1": 1}[n]
    opts = {"path": ak.AK_PATH_BLOCK}
    keys = synth.random_keys(n, dtype, seed=60 + n, mode="dups" if n % 2 else "bits")
    for desc in (False, True):
        order = "descending" if desc else "ascending"
        p = oracle_perm(keys, desc)
        t, u = to_dev(keys)
        ak.ak_sort(t, order, options=opts, unsigned=u)
        assert_bits_equal(to_host(t, keys.dtype), oracle.gather(keys, p), "block sort")
        t, u = to_dev(keys)
        perm = ak.ak_sortperm(t, order, options=opts, unsigned=u)
        assert np.array_equal(to_host(perm, np.uint32), p.astype(np.uint32))
        assert_bits_equal(to_host(t, keys.dtype), keys, "sortperm keys untouched")
        vals = np.arange(n, dtype=np.uint64) * np.uint64(3)
        t, u = to_dev(keys)
        v, _ = to_dev(vals)
        ak.ak_sort_pairs(t, v, order, options=opts, unsigned=u)
        assert_bits_equal(to_host(v, np.uint64), vals[p], "block pairs")


def test_auto_picks_block_merge_radix_by_size(ak):
    keys = synth.random_keys(3000, np.uint32, seed=1)
    t, u = to_dev(keys)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, 3000, ak.AK_U32), t.device)
    ak.ak_sort(t, temp=temp, unsigned=u)
    assert ak.ak_last_info(temp)["path"] == ak.AK_PATH_BLOCK
    keys = synth.random_keys(300000, np.uint32, seed=1)
    t, u = to_dev(keys)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, keys.size, ak.AK_U32), t.device)
    ak.ak_sort(t, temp=temp, unsigned=u)
    assert ak.ak_last_info(temp)["path"] == ak.AK_PATH_RADIX
    # a few capacity tiles: the merge path, exact
    n = 5 * ak.ak_segment_capacity(4, 0) + 17
    keys = synth.random_keys(n, np.uint32, seed=2)
    t, u = to_dev(keys)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_U32), t.device)
    ak.ak_sort(t, temp=temp, unsigned=u)
    assert ak.ak_last_info(temp)["path"] == ak.AK_PATH_MERGE
    assert np.array_equal(to_host(t, np.uint32), np.sort(keys))


@pytest.mark.parametrize("dtype", [np.uint16, np.int32, np.float32, np.uint64, np.float64])
@pytest.mark.parametrize("tiles", [1.5, 2, 3.2, 8, 8.01, 77.3])
def test_merge_path_sort_perm_pairs(ak, dtype, tiles):
    """AK_PATH_MERGE: tiles of the shared-memory capacity sorted in one launch,
    then stable merge-path rounds (odd and even round counts, ragged last runs)."""
    kb = np.dtype(dtype).itemsize
    cap = ak.ak_segment_capacity(kb, 0)
    n = int(tiles * cap)
    opts = {"path": ak.AK_PATH_MERGE}
    keys = synth.random_keys(n, dtype, seed=int(tiles * 100) + kb, mode="dups" if tiles in (2, 8.01) else "bits")
    for desc in (False, True):
        order = "descending" if desc else "ascending"
        p = oracle_perm(keys, desc)
        t, u = to_dev(keys)
        temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, n, ak.dtype_code(t, u), options=opts), t.device)
        ak.ak_sort(t, order, temp=temp, options=opts, unsigned=u)
        assert ak.ak_last_info(temp)["path"] == ak.AK_PATH_MERGE
        assert_bits_equal(to_host(t, keys.dtype), oracle.gather(keys, p), "merge sort")
        t, u = to_dev(keys)
        perm = ak.ak_sortperm(t, order, options=opts, unsigned=u)
        assert np.array_equal(to_host(perm, np.uint32), p.astype(np.uint32)), "merge sortperm"
        vals = (np.arange(n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)).astype(np.uint16)
        t, u = to_dev(keys)
        v, _ = to_dev(vals)
        ak.ak_sort_pairs(t, v, order, options=opts, unsigned=u)
        assert_bits_equal(to_host(v, np.uint16), vals[p], "merge pairs")
