"""Parity of the benchmark configurations at their full sizes, through the C ABI.

* the key-value configuration: 2^30 u32 keys, half Zipf(s=1.1) over 2^24 ranks
  and half uniform, u32 values = input index, descending ak_sort_pairs, through
  the plain radix path and the learned-bucket path (with its fallback); bit-exact
  against the oracle at 2^24 keys, and at 2^30 through the stable-permutation
  properties (values = input index make the permutation observable);
* the segmented batch: all 65,536 lognormal segments (269M u32 keys), one
  persistent launch replayed from a CUDA graph, every segment against its own
  sort;
* the six float64 distributions at 1e8 keys, learned and plain, sortperm checked
  through the stable-permutation properties and sort = keys[perm] bit for bit;
* n > 2^30: the 64-bit look-back words of the digit pass (u16 keys, whose exact
  sorted output is the counting sort of their 65,536 values).

Expected values come from the oracle, or from properties that characterise the
unique stable result (pinned against the oracle by the CPU tests).  This file
runs after the other parity files: its inputs are large.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_bits_equal, check_perm_properties, oracle_perm, to_dev, to_host

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _pairs(ak, keys, vals, path):
    """Descending ak_sort_pairs through `path`; returns (keys, values, ak_info)."""
    opts = {"path": path}
    kt, ku = to_dev(keys)
    vt, _ = to_dev(vals)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT_PAIRS, keys.size, ak.dtype_code(kt, ku), 4, options=opts),
                        kt.device)
    ak.ak_sort_pairs(kt, vt, "descending", temp=temp, options=opts, unsigned=ku)
    info = ak.ak_last_info(temp)
    k_out, v_out = to_host(kt, keys.dtype), to_host(vt, vals.dtype)
    del kt, vt, temp
    torch.cuda.empty_cache()
    return k_out, v_out, info


def test_small_zipf_mix_matches_oracle_both_orders(ak):
    """A quick case of the same key distribution (both orders, both paths,
    keys only) so that a failure shows before the large cases run."""
    n = 300_007
    keys = synth.zipf_mix_u32(n, seed=31)
    for desc in (False, True):
        p = oracle_perm(keys, desc)
        for path in (ak.AK_PATH_RADIX, ak.AK_PATH_LEARNED):
            t, u = to_dev(keys)
            ak.ak_sort(t, "descending" if desc else "ascending", options={"path": path}, unsigned=u)
            torch.cuda.synchronize()
            assert_bits_equal(to_host(t, np.uint32), oracle.gather(keys, p), f"path {path} desc={desc}")


@pytest.mark.parametrize("path", ["radix", "learned"])
def test_zipf_mix_pairs_descending_exact(ak, path):
    """2^24 keys of the key-value configuration's distribution, bit-exact
    against the oracle's stable descending key-value sort."""
    n = 1 << 24
    keys = synth.zipf_mix_u32(n, seed=30, workers=min(THREADS, 8))
    vals = np.arange(n, dtype=np.uint32)
    want_k, want_v = oracle.sort_pairs(keys, vals, "descending", threads=THREADS)
    p = {"radix": ak.AK_PATH_RADIX, "learned": ak.AK_PATH_LEARNED}[path]
    got_k, got_v, info = _pairs(ak, keys, vals, p)
    assert info["status"] == 0
    assert_bits_equal(got_k, want_k, "zipf-mix pair keys")
    assert_bits_equal(got_v, want_v, "zipf-mix pair values")


@pytest.mark.slow
@pytest.mark.parametrize("path", ["radix", "learned"])
def test_zipf_mix_pairs_descending_full_size(ak, path):
    """The key-value configuration at full size: 2^30 keys with their input
    index as value (8 GiB).  The values returned are the sorting permutation:
    it must be THE stable descending sortperm, and the keys must be keys[perm]."""
    n = 1 << 30
    keys = synth.zipf_mix_u32(n, seed=30, workers=THREADS)
    vals = np.arange(n, dtype=np.uint32)
    p = {"radix": ak.AK_PATH_RADIX, "learned": ak.AK_PATH_LEARNED}[path]
    got_k, got_v, info = _pairs(ak, keys, vals, p)
    assert info["status"] == 0
    del vals
    check_perm_properties(keys, got_v, descending=True)
    assert_bits_equal(got_k, keys[got_v.astype(np.int64)], "full-size pair keys = keys[perm]")


@pytest.mark.slow
def test_segmented_full_batch_graph_replay(ak):
    """All 65,536 lognormal segments (median 2,048, clipped to [1, 2^20]),
    269M uniform u32 keys, sorted by one persistent launch replayed from a CUDA
    graph.  Equal u32 keys are bit-identical, so each segment's stable sort is
    its numpy sort; (segment id, key) sorted as one 64-bit word gives all of
    them at once."""
    off = synth.lognormal_segments(65536, seed=20)
    n = int(off[-1])
    keys = synth.uniform_u32(n, seed=21)
    t, u = to_dev(keys)
    pristine = t.clone()
    o = torch.from_numpy(off).cuda()
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT_SEGMENTED, n, ak.AK_U32, nseg=off.size - 1), t.device)
    s = torch.cuda.Stream()
    ak.ak_sort_segmented(t, o, temp=temp, stream=s, unsigned=u)  # outside capture: kernel attributes
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ak.ak_sort_segmented(t, o, temp=temp, stream=s, unsigned=u)
    for _ in range(2):
        t.copy_(pristine)
        g.replay()
    torch.cuda.synchronize()
    got = to_host(t, np.uint32)
    assert ak.ak_status_check(temp) == 0
    del t, pristine, temp, g
    torch.cuda.empty_cache()
    seg = np.repeat(np.arange(off.size - 1, dtype=np.uint64), np.diff(off))
    want = np.sort((seg << np.uint64(32)) | keys.astype(np.uint64)).astype(np.uint32)
    assert_bits_equal(got, want, "full segmented batch")


@pytest.mark.slow
@pytest.mark.parametrize("dist", synth.F64_DISTS)
def test_six_distributions_1e8_learned_and_plain(ak, dist):
    """1e8 float64 keys of each distribution through the learned path and the
    plain radix path: sortperm is THE stable sortperm, sort = keys[perm]."""
    n = 100_000_000
    keys = synth.dist_f64(n, dist, seed=10 + synth.F64_DISTS.index(dist))
    for path in (ak.AK_PATH_LEARNED, ak.AK_PATH_RADIX):
        opts = {"path": path}
        t, _ = to_dev(keys)
        temp = ak.workspace(max(ak.temp_bytes(op, n, ak.AK_F64, options=opts)
                                for op in (ak.AK_OP_SORT, ak.AK_OP_SORTPERM)), t.device)
        p = ak.ak_sortperm(t, temp=temp, options=opts)
        assert ak.ak_status_check(temp) == 0
        perm = to_host(p, np.uint32)
        del p
        check_perm_properties(keys, perm, descending=False)
        ak.ak_sort(t, temp=temp, options=opts)
        info = ak.ak_last_info(temp)
        assert info["status"] == 0
        if path == ak.AK_PATH_LEARNED and dist in ("uniform", "normal", "presorted", "reversed"):
            assert info["path"] == ak.AK_PATH_LEARNED, (dist, info)
        assert_bits_equal(to_host(t, np.float64), keys[perm.astype(np.int64)], f"{dist} sort = keys[perm]")
        del t, temp
        torch.cuda.empty_cache()


@pytest.mark.slow
def test_wide_lookback_words_above_2_30(ak):
    """n = 2^30 + 4,097 u16 keys: the digit pass keeps 62-bit counts in 64-bit
    look-back words (n > 2^30).  The stable sort of u16 keys is their counting
    sort; sortperm is checked through the stable-permutation properties."""
    n = (1 << 30) + 4097
    keys = synth.random_keys(n, np.uint16, seed=61, mode="bits")
    counts = np.bincount(keys, minlength=1 << 16)
    rad = {"path": ak.AK_PATH_RADIX}
    for desc in (False, True):
        t, u = to_dev(keys)
        ak.ak_sort(t, "descending" if desc else "ascending", options=rad, unsigned=u)
        torch.cuda.synchronize()
        got = to_host(t, np.uint16)
        del t
        values = np.arange(1 << 16, dtype=np.uint16)
        want = np.repeat(values[::-1], counts[::-1]) if desc else np.repeat(values, counts)
        assert_bits_equal(got, want, f"u16 counting sort, desc={desc}")
        del got, want
    t, u = to_dev(keys)
    p = ak.ak_sortperm(t, options=rad, unsigned=u)
    torch.cuda.synchronize()
    perm = to_host(p, np.uint32)
    del p
    check_perm_properties(keys, perm, descending=False)
    p = ak.ak_sortperm_lowmem(t, unsigned=u)  # the gather passes with 64-bit look-back words
    torch.cuda.synchronize()
    assert np.array_equal(to_host(p, np.uint32), perm), "lowmem sortperm differs from sortperm"
    del p, t
    torch.cuda.empty_cache()
