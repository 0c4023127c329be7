"""ak_sort_static_scratch: the sort for callers that cannot allocate device
memory (its workspace is a static array inside the library).

Its output must equal ak_sort's (the entry point with a caller workspace)
bit for bit, on two calls in a row that share the static array.  This file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _call_static(lib, t, kd):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.ak_sort_static_scratch(ctypes.c_void_p(t.data_ptr()), t.numel(), kd, 0, ctypes.c_void_p(stream))


def test_static_scratch_matches_ak_sort_twice(ak):
    lib = ak.load()
    cases = [
        (synth.normal_f32_special(1_000_003, seed=91, frac=0.01), ak.AK_F32),   # radix path
        (synth.uniform_i64(300_001, seed=92), ak.AK_I64),                       # radix path, 8 passes
        (synth.random_keys(2_000, np.float64, seed=93, mode="dups"), ak.AK_F64),  # one-launch block path
    ]
    for keys, kd in cases:
        for rep in range(2):  # two calls in a row share the static array
            a = torch.from_numpy(keys.copy()).cuda()
            b = a.clone()
            assert _call_static(lib, a, kd) == 0
            ak.ak_sort(b)  # the entry point with a caller workspace
            torch.cuda.synchronize()
            assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), (keys.dtype, rep)


def test_static_scratch_rejects_oversized_requests(ak):
    lib = ak.load()
    t = torch.zeros(16, dtype=torch.int64, device="cuda")
    # a request whose workspace exceeds the static array is refused before any launch
    rc = lib.ak_sort_static_scratch(ctypes.c_void_p(t.data_ptr()), 1 << 28, ak.AK_I64, 0, None)
    assert rc == 3  # AK_ERR_WORKSPACE_TOO_SMALL
    assert torch.count_nonzero(t).item() == 0
