"""Autotuner on the GPU: it picks one of its candidates, leaves the inputs as
they were, and AK_PATH_AUTO calls then take its choice and stay exact."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_bits_equal, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


@pytest.mark.parametrize("op", ["sort", "sortperm", "pairs"])
def test_autotune_then_auto_call(ak, op):
    ak.ak_autotune_clear()
    keys = synth.dist_f64(1 << 20, "normal", seed=4)
    t, _ = to_dev(keys)
    vals = perm = None
    code = {"sort": ak.AK_OP_SORT, "sortperm": ak.AK_OP_SORTPERM, "pairs": ak.AK_OP_SORT_PAIRS}[op]
    if op == "pairs":
        vals = torch.arange(keys.size, dtype=torch.int32, device="cuda")
    if op == "sortperm":
        perm = torch.empty(keys.size, dtype=torch.int32, device="cuda")
    best = ak.ak_autotune(code, t, vals=vals, perm=perm)
    assert best.path in (ak.AK_PATH_RADIX, ak.AK_PATH_LEARNED, ak.AK_PATH_BLOCK)
    assert_bits_equal(to_host(t, np.float64), keys, "inputs restored")
    temp = ak.workspace(ak.temp_bytes(code, keys.size, ak.AK_F64, 4 if op == "pairs" else 0), t.device)
    p = oracle.sortperm(keys)
    if op == "sort":
        ak.ak_sort(t, temp=temp)
        assert_bits_equal(to_host(t, np.float64), keys[p], "sort")
    elif op == "sortperm":
        out = ak.ak_sortperm(t, temp=temp)
        assert np.array_equal(to_host(out, np.uint32), p.astype(np.uint32))
    else:
        ak.ak_sort_pairs(t, vals, temp=temp)
        assert np.array_equal(vals.cpu().numpy(), p.astype(np.int32))
    assert ak.ak_last_info(temp)["path"] in (best.path, ak.AK_PATH_RADIX)
    ak.ak_autotune_clear()


def test_autotune_segmented_picks_a_split_threshold_and_stays_exact(ak):
    """The segmented tuner times the split thresholds on a lognormal batch,
    restores the keys, caches its choice; the next default call takes it and
    every segment is sorted."""
    ak.ak_autotune_clear()
    off = synth.lognormal_segments(4096, seed=20)
    n = int(off[-1])
    keys = synth.uniform_u32(n, seed=21)
    t, u = to_dev(keys)
    o = torch.from_numpy(off).cuda()
    best = ak.ak_autotune_segmented(t, o, unsigned=u)
    assert best.split_caps in (1, 2, 4, 8, 16, -1)
    assert_bits_equal(to_host(t, np.uint32), keys, "inputs restored")
    ak.ak_sort_segmented(t, o, unsigned=u)
    torch.cuda.synchronize()
    seg = np.repeat(np.arange(off.size - 1, dtype=np.uint64), np.diff(off))
    want = np.sort((seg << np.uint64(32)) | keys.astype(np.uint64)).astype(np.uint32)
    assert_bits_equal(to_host(t, np.uint32), want, "tuned segmented sort")
    ak.ak_autotune_clear()


@pytest.mark.parametrize("caps", [1, 2, 16, -1])
def test_every_split_threshold_is_exact(ak, caps):
    off = synth.lognormal_segments(1024, seed=23, median=8192.0)
    n = int(off[-1])
    keys = synth.random_keys(n, np.float32, seed=24, mode="bits")
    t, u = to_dev(keys)
    ak.ak_sort_segmented(t, torch.from_numpy(off).cuda(), options={"split_caps": caps}, unsigned=u)
    torch.cuda.synchronize()
    want = oracle.sort_segmented(keys, off)
    assert_bits_equal(to_host(t, np.float32), want, f"split_caps {caps}")
