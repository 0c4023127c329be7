"""ak_sort_static_scratch: the sort for callers that cannot allocate device
memory (its workspace is a static array inside the library).

Its output must equal the oracle's sort, and ak_sort's (the entry point with a
caller workspace) bit for bit, on two calls in a row that share the static
array.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

STATIC_BYTES = 32 << 20  # AK_STATIC_SCRATCH_BYTES


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _call_static(lib, t, kd, n=None, desc=False):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.ak_sort_static_scratch(ctypes.c_void_p(t.data_ptr()), t.numel() if n is None else n, kd,
                                      1 if desc else 0, ctypes.c_void_p(stream))


def _largest_fitting_n(ak, kd):
    """Largest n whose ak_sort workspace (default options) fits the static array."""
    lo, hi = 1, 1 << 26
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if ak.temp_bytes(ak.AK_OP_SORT, mid, kd) <= STATIC_BYTES:
            lo = mid
        else:
            hi = mid - 1
    return lo


def test_static_scratch_matches_oracle_and_ak_sort_twice(ak):
    lib = ak.load()
    cases = [
        (synth.normal_f32_special(1_000_003, seed=91, frac=0.01), ak.AK_F32),   # radix path
        (synth.uniform_i64(300_001, seed=92), ak.AK_I64),                       # radix path, 8 passes
        (synth.random_keys(2_000, np.float64, seed=93, mode="dups"), ak.AK_F64),  # one-launch block path
    ]
    for keys, kd in cases:
        for desc in (False, True):
            want = oracle.sort(keys, "descending" if desc else "ascending")
            for rep in range(2):  # two calls in a row share the static array
                a = torch.from_numpy(keys.copy()).cuda()
                b = a.clone()
                assert _call_static(lib, a, kd, desc=desc) == 0
                ak.ak_sort(b, "descending" if desc else "ascending")  # the entry point with a caller workspace
                torch.cuda.synchronize()
                got = a.cpu().numpy()
                assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (keys.dtype, desc, rep)
                assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), (keys.dtype, desc, rep)


def test_static_scratch_largest_size_and_refusal(ak):
    """The largest n whose workspace fits is sorted exactly; one key more is
    refused before any launch (the keys stay untouched)."""
    lib = ak.load()
    for np_dt, kd in ((np.uint32, ak.AK_U32), (np.int64, ak.AK_I64)):
        n = _largest_fitting_n(ak, kd)
        assert ak.temp_bytes(ak.AK_OP_SORT, n + 1, kd) > STATIC_BYTES
        keys = synth.random_keys(n + 1, np_dt, seed=94, mode="bits")
        t = torch.from_numpy(keys.view(np.int32 if np_dt == np.uint32 else np.int64).copy()).cuda()
        assert lib.ak_sort_static_scratch(ctypes.c_void_p(t.data_ptr()), n + 1, kd, 0, None) == 3
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy().view(np_dt), keys), "refused call touched the keys"
        assert _call_static(lib, t, kd, n=n) == 0
        torch.cuda.synchronize()
        got = t.cpu().numpy().view(np_dt)
        assert np.array_equal(got[:n], oracle.sort(keys[:n])), np_dt
        assert got[n] == keys[n]


def test_static_scratch_allocates_nothing(ak):
    """After the first call on the device (which looks up the array's address),
    further calls change neither torch's allocation nor the device's free memory."""
    lib = ak.load()
    keys = synth.uniform_i64(500_000, seed=95)
    t = torch.from_numpy(keys.copy()).cuda()
    assert _call_static(lib, t, ak.AK_I64) == 0
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        t.copy_(torch.from_numpy(keys))
        assert _call_static(lib, t, ak.AK_I64) == 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(t.cpu().numpy(), np.sort(keys))


def test_static_scratch_rejects_oversized_requests(ak):
    lib = ak.load()
    t = torch.zeros(16, dtype=torch.int64, device="cuda")
    # a request whose workspace exceeds the static array is refused before any launch
    rc = lib.ak_sort_static_scratch(ctypes.c_void_p(t.data_ptr()), 1 << 28, ak.AK_I64, 0, None)
    assert rc == 3  # AK_ERR_WORKSPACE_TOO_SMALL
    assert torch.count_nonzero(t).item() == 0
