"""16-bit float keys (IEEE binary16 and bfloat16) through every sort path and
the binary search, bit-exact against the oracle (which decodes both exactly to
float32 and orders them by Julia isless: -0.0 before +0.0, every NaN last and
tied, NaN payloads kept in input order)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_bits_equal

pytestmark = pytest.mark.gpu

BF16_SPECIALS = np.array([0x0000, 0x8000, 0x7F80, 0xFF80, 0x7FC0, 0xFFC1, 0x7FC5, 0x7F81, 0x0001, 0x8001,
                          0x3F80, 0xBF80, 0x7F7F, 0xFF7F, 0x0080, 0x8080], dtype=np.uint16)


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _keys(kind, n, seed, mode):
    """u16 bit patterns of the keys."""
    if mode == "bits":
        return (synth.splitmix64(seed, n) >> np.uint64(48)).astype(np.uint16)
    if kind == "f16":
        pool = np.concatenate([synth.special_values(np.float16).view(np.uint16),
                               (synth.splitmix64(seed + 1, 40) >> np.uint64(48)).astype(np.uint16)])
    else:
        pool = np.concatenate([BF16_SPECIALS, (synth.splitmix64(seed + 1, 40) >> np.uint64(48)).astype(np.uint16)])
    if mode == "narrow":  # one exponent band: the upper radix digit is the same for most keys
        base = np.uint16(0x3C00 if kind == "f16" else 0x3F80)
        return (base | (synth.splitmix64(seed, n) % np.uint64(128)).astype(np.uint16)).astype(np.uint16)
    return pool[(synth.splitmix64(seed + 2, n) % np.uint64(pool.size)).astype(np.int64)]


def _perm(kind, bits, desc):
    order = "descending" if desc else "ascending"
    if kind == "f16":
        return oracle.sortperm(bits.view(np.float16), order)
    return oracle.sortperm(bits, order, as_dtype="bfloat16")


def _dev(kind, bits):
    t = torch.from_numpy(bits.view(np.int16).copy()).cuda()
    return t.view(torch.float16 if kind == "f16" else torch.bfloat16)


def _host(t):
    return t.view(torch.int16).cpu().numpy().view(np.uint16)


PATHS = {"radix": 1, "learned": 2, "block": 3, "merge": 4, "auto": 0}


@pytest.mark.parametrize("kind", ["f16", "bf16"])
@pytest.mark.parametrize("mode", ["bits", "dups", "narrow"])
@pytest.mark.parametrize("path", ["radix", "learned", "auto"])
def test_sort_sortperm_pairs(ak, kind, mode, path):
    opts = {"path": PATHS[path]}
    for n in (1, 1000, 5761, 100_003):
        bits = _keys(kind, n, seed=500 + n, mode=mode)
        for desc in (False, True):
            order = "descending" if desc else "ascending"
            p = _perm(kind, bits, desc)
            t = _dev(kind, bits)
            ak.ak_sort(t, order, options=opts)
            torch.cuda.synchronize()
            assert_bits_equal(_host(t), bits[p], f"{kind} {mode} {path} sort n={n} desc={desc}")
            t = _dev(kind, bits)
            perm = ak.ak_sortperm(t, order, options=opts)
            torch.cuda.synchronize()
            assert np.array_equal(perm.cpu().numpy().view(np.uint32), p.astype(np.uint32)), (kind, n, desc)
            vals = np.arange(n, dtype=np.int32)
            t, v = _dev(kind, bits), torch.from_numpy(vals).cuda()
            ak.ak_sort_pairs(t, v, order, options=opts)
            torch.cuda.synchronize()
            assert np.array_equal(v.cpu().numpy(), p.astype(np.int32)), (kind, n, desc, "pairs")
            assert_bits_equal(_host(t), bits[p], "pair keys")


@pytest.mark.parametrize("kind", ["f16", "bf16"])
@pytest.mark.parametrize("path", ["block", "merge"])
def test_block_and_merge_paths(ak, kind, path):
    cap = ak.ak_segment_capacity(2, 0)
    for n in ((7, cap - 1, cap) if path == "block" else (cap + 1, 3 * cap + 17)):
        bits = _keys(kind, n, seed=600 + n, mode="dups")
        for desc in (False, True):
            p = _perm(kind, bits, desc)
            t = _dev(kind, bits)
            ak.ak_sort(t, "descending" if desc else "ascending", options={"path": PATHS[path]})
            torch.cuda.synchronize()
            assert_bits_equal(_host(t), bits[p], f"{kind} {path} n={n}")


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_segmented(ak, kind):
    lens = [0, 1, 2, 33, 500, 9000, 50_000, 3, 200_000]
    off = np.zeros(len(lens) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    bits = _keys(kind, int(off[-1]), seed=700, mode="bits")
    as_dtype = None if kind == "f16" else "bfloat16"
    src = bits.view(np.float16) if kind == "f16" else bits
    for desc in (False, True):
        order = "descending" if desc else "ascending"
        want = bits[oracle.sortperm_segmented(src, off, order, as_dtype=as_dtype)]
        t = _dev(kind, bits)
        ak.ak_sort_segmented(t, torch.from_numpy(off).cuda(), order)
        torch.cuda.synchronize()
        assert_bits_equal(_host(t), want, f"{kind} segmented desc={desc}")


@pytest.mark.parametrize("kind", ["f16", "bf16"])
@pytest.mark.parametrize("desc", [False, True])
def test_searchsorted(ak, kind, desc):
    order = "descending" if desc else "ascending"
    bits = _keys(kind, 50_001, seed=800, mode="dups")
    v = bits[_perm(kind, bits, desc)]
    x = np.concatenate([_keys(kind, 20_000, seed=801, mode="bits"), v[::7]])
    as_dtype = None if kind == "f16" else "bfloat16"
    vv = v.view(np.float16) if kind == "f16" else v
    xx = x.view(np.float16) if kind == "f16" else x
    for side, fn in (("first", ak.ak_searchsortedfirst), ("last", ak.ak_searchsortedlast)):
        want = oracle.searchsorted(vv, xx, side, order, as_dtype=as_dtype)
        got = fn(_dev(kind, v), _dev(kind, x), order).cpu().numpy()
        assert np.array_equal(got, want), (kind, desc, side)


def test_accumulate_refuses_16bit_floats(ak):
    t = torch.ones(16, dtype=torch.float16, device="cuda")
    with pytest.raises(ak.AkError) as e:
        ak.ak_accumulate(t)
    assert e.value.status == 2
