"""Parity of accumulate (Sec. II-B prefix scan) against the CPU oracle through
the C ABI: bit-exact for integers and max/min (any NaN for a NaN); for float +
within the rounding bound of the kernel's summation depth."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import to_dev, to_host

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


def _scan(ak, x, op, inclusive, init=None, offset=0):
    """Scan through the C ABI; `offset` elements shift both arrays off 16-byte alignment."""
    t, u = to_dev(np.concatenate([np.zeros(offset, x.dtype), x]))
    o = torch.empty_like(t)
    got = ak.ak_accumulate(t[offset:], op, inclusive, init=init, out=o[offset:], unsigned=u)
    torch.cuda.synchronize()
    return to_host(got, x.dtype)


def _float_add_bound(x, init, dtype):
    """Rounding bound of any summation tree of depth D over the prefix terms:
    gamma_D * (|init| + sum |x_j|), D = m + 2 ceil(n / (32768 m)) + 84 with m
    keys per lane and warp tile (64 bytes of keys, 32 for 16-bit keys; at
    least 1,024 warp ranges once there are that many tiles), plus one ulp for
    the oracle's own single rounding to the key type."""
    w = np.dtype(dtype).itemsize
    m = 16 if w == 2 else 64 // w
    d = m + 2 * -(-x.size // (32768 * m)) + 84
    u = np.finfo(dtype).eps / 2
    gamma = d * u / (1 - d * u)
    s = abs(float(init)) + np.cumsum(np.abs(x.astype(np.float64)))
    return gamma * s


def _check(got, want, x, op, init, dtype):
    if np.dtype(dtype).kind == "f":
        gn, wn = np.isnan(got), np.isnan(want)
        assert np.array_equal(gn, wn), "NaN positions differ"
        g, w = got[~gn], want[~wn]
        if op == "add":
            tol = _float_add_bound(x, init, dtype)[~wn] + np.spacing(np.abs(w).astype(dtype)).astype(np.float64)
            err = np.abs(g.astype(np.float64) - w.astype(np.float64))
            same_inf = np.isinf(g) & (g == w)
            bad = ~same_inf & ~(err <= tol)
            assert not bad.any(), f"{bad.sum()} outside the bound, first at {np.flatnonzero(bad)[0]}"
            return
        got, want = g, w
    u = np.dtype(f"u{np.dtype(dtype).itemsize}")
    assert np.array_equal(np.ascontiguousarray(got).view(u), np.ascontiguousarray(want).view(u))


def _keys(dtype, n, seed, op):
    """Integers: all bit patterns (+ wraps); floats for +: finite, mixed signs and
    magnitudes; floats for max/min: duplicates and every special value."""
    if np.dtype(dtype).kind == "f" and op == "add":
        u = synth.u01_f64(seed, n)
        mag = np.exp2(np.floor(synth.u01_f64(seed + 1, n) * 30) - 15)
        return ((u - 0.5) * mag).astype(dtype)
    return synth.random_keys(n, dtype, seed, mode="dups" if np.dtype(dtype).kind == "f" else "bits")


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("op", ["add", "max", "min"])
@pytest.mark.parametrize("inclusive", [True, False])
def test_parity_all_dtypes(ak, dtype, op, inclusive):
    """100,003 keys: hundreds of warp tiles, one range each, the last one ragged; a start value."""
    x = _keys(dtype, 100_003, 111, op)
    init = np.array([5]).astype(dtype)[0] if op == "add" else oracle.identity(dtype, op)
    got = _scan(ak, x, op, inclusive, init=init)
    _check(got, oracle.accumulate(x, op, inclusive, init), x, op, init, dtype)


@pytest.mark.parametrize("dtype", [np.uint16, np.int32, np.float32, np.float64])
def test_sizes_alignment_and_in_place(ak, dtype):
    """n = 1, a lane's run, a warp tile -1/+0/+1, 1,024 warp tiles + 3 (one
    per range) and 6,000 + 7 (several per range, ragged); pointers off
    16-byte alignment (scalar loads); the in-place form."""
    w = np.dtype(dtype).itemsize
    wt = 32 * (16 if w == 2 else 64 // w)  # keys per warp tile: 64 bytes a lane, 32 for 16-bit keys
    for n in (1, 2, 31, wt - 1, wt, wt + 1, 1024 * wt + 3, 6000 * wt + 7):
        x = _keys(dtype, n, 112 + n, "add")
        for offset in (0, 1):
            for inclusive in (True, False):
                got = _scan(ak, x, "add", inclusive, offset=offset)
                init = oracle.identity(dtype, "add")
                _check(got, oracle.accumulate(x, "add", inclusive, init), x, "add", init, dtype)
        y = _keys(dtype, n, 113 + n, "max")
        t, u = to_dev(y)
        r = ak.ak_accumulate(t, "max", out=t, unsigned=u)  # in place
        torch.cuda.synchronize()
        assert r is t
        _check(to_host(t, y.dtype), oracle.accumulate(y, "max"), y, "max", None, dtype)


def test_float_add_specials(ak):
    """IEEE + with Inf and NaN in the prefix: order does not matter for these."""
    x = np.full(50_000, 0.25, dtype=np.float32)
    x[1000] = np.inf
    got = _scan(ak, x, "add", True)
    assert np.all(got[:1000] == np.cumsum(x[:1000])) and np.all(np.isposinf(got[1000:]))
    x[30_000] = -np.inf
    got = _scan(ak, x, "add", True)
    assert np.all(np.isposinf(got[1000:30_000])) and np.all(np.isnan(got[30_000:]))
    z = np.full(20_000, -0.0)
    got = _scan(ak, z, "add", True)  # the identity start: sums of -0.0 stay -0.0
    assert np.all(np.signbit(got))
    got = _scan(ak, z, "add", False, init=-0.0)
    assert np.all(np.signbit(got)) and got.size == z.size


def test_empty_and_default_start_values(ak):
    t = torch.empty(0, dtype=torch.int32, device="cuda")
    assert ak.ak_accumulate(t).numel() == 0
    x = np.array([4, -7, 2], dtype=np.int16)
    assert _scan(ak, x, "max", False).tolist() == [-32768, 4, 4]
    assert _scan(ak, x, "min", False).tolist() == [32767, 4, -7]
    assert _scan(ak, x, "add", False, init=10).tolist() == [10, 14, 7]


def test_wait_options_are_inert(ak):
    """No kernel of the scan waits on another CTA: the timeout and the
    skip-first-tile hook change nothing, the status stays AK_OK and the
    result is exact."""
    n = 20 * 4096 + 5
    x = synth.random_keys(n, np.int32, seed=77, mode="bits")
    t, _ = to_dev(x)
    temp = ak.workspace(ak.accumulate_temp_bytes(n, ak.AK_I32), t.device)
    opts = {"timeout_ns": 1, "debug_flags": ak.AK_DEBUG_SKIP_FIRST_TILE}
    got = ak.ak_accumulate(t, out=torch.empty_like(t), temp=temp, options=opts)
    assert ak.ak_status_check(temp) == 0
    _check(to_host(got, np.int32), oracle.accumulate(x, "add", True), x, "add", 0, np.int32)
