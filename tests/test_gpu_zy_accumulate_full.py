"""Accumulate at full size (2^28 keys), the shapes the benchmark times.  Kept
in a file of its own that runs after the other GPU parity files."""
import numpy as np
import pytest
import torch

import oracle
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


@pytest.mark.slow
def test_full_size(ak):
    """268,435,456 int64 keys (2 GiB) scanned with + (every output exact), and
    268,435,456 float32 keys holding small integers, where every output is
    exact too: any node of any summation tree is a sum of consecutive keys,
    at most max(S) - min(S) in size (S the prefix sums, 0 included), and
    below 2^24 every such float32 sum is an exact integer -- so the scan's
    order cannot change a bit.  The shapes the benchmark times."""
    n = 1 << 28
    x = synth.uniform_i64(n, seed=114)
    t = torch.from_numpy(x).cuda()
    got = ak.ak_accumulate(t).cpu().numpy()
    assert np.array_equal(got, oracle.accumulate(x, "add"))
    del t, got, x
    xi = (synth.splitmix64(115, n) % np.uint64(17)).astype(np.int64) - 8  # integers -8 .. 8
    s = np.cumsum(xi)
    assert max(int(s.max()), 0) - min(int(s.min()), 0) < (1 << 24)  # the exactness condition
    tf = torch.from_numpy(xi.astype(np.float32)).cuda()
    gf = ak.ak_accumulate(tf).cpu().numpy()
    assert np.array_equal(gf, s.astype(np.float32))
    want = oracle.accumulate(xi.astype(np.float32), "add")
    assert np.array_equal(gf, want)
