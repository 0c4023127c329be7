"""Accumulate at full size (2^28 keys), the shapes the benchmark times.  Kept
in a file of its own that runs after the other GPU parity files."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.test_gpu_accumulate import _float_add_bound, _keys

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


@pytest.mark.slow
def test_full_size(ak):
    """268,435,456 int64 keys (2 GiB) scanned with + (every output exact), and
    268,435,456 float32 keys with + against the bound on 20,000 sampled outputs
    -- the shapes and launch configuration the benchmark times."""
    n = 1 << 28
    x = synth.uniform_i64(n, seed=114)
    t = torch.from_numpy(x).cuda()
    got = ak.ak_accumulate(t).cpu().numpy()
    assert np.array_equal(got, np.cumsum(x, dtype=np.int64))
    del t
    xf = _keys(np.float32, n, 115, "add")
    tf = torch.from_numpy(xf).cuda()
    gf = ak.ak_accumulate(tf).cpu().numpy()
    want = oracle.accumulate(xf, "add")
    pick = np.sort((synth.splitmix64(116, 20_000) % np.uint64(n)).astype(np.int64))
    bound = _float_add_bound(xf, 0.0, np.float32)[pick] + np.spacing(np.abs(want[pick]))
    assert np.all(np.abs(gf[pick].astype(np.float64) - want[pick].astype(np.float64)) <= bound)
