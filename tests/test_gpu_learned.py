"""Learned-CDF bucketing path: model kernels against the float64 restatement,
and every sorted output bit-exact against the merge-sort oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import learned as L
import synth
from tests.gpu_util import assert_bits_equal, oracle_perm, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ak():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as m
    return m


def _learned(ak, **kw):
    o = {"path": ak.AK_PATH_LEARNED}
    o.update(kw)
    return o


def test_knots_exact(ak):
    """Knots are sample order statistics: bit-exact against the restatement."""
    for seed, m in ((1, 1), (2, 64), (3, 1000), (4, 65537), (5, 1 << 20)):
        xs = np.sort(synth.u01_f64(seed, m).astype(np.float32))
        got = ak.ak_learned_knots(torch.from_numpy(xs).cuda()).cpu().numpy()
        assert np.array_equal(got.view(np.uint32), L.pl_knots(xs).view(np.uint32)), seed


@pytest.mark.parametrize("seed", [11, 12])
def test_loss_and_gradient_match_float64(ak, seed):
    m = 5000
    x = np.sort(synth.u01_f64(seed, m)).astype(np.float32)
    y = ((np.arange(m) + 0.5) / m).astype(np.float32)
    c = np.sort(synth.u01_f64(seed + 1, L.N_KNOTS)).astype(np.float32)  # knots xi
    p = ((synth.u01_f64(seed + 2, L.N_PARAMS) - 0.5) * 0.8).astype(np.float32)
    p[L.P_W3:L.P_B3 + 1] *= 64.0  # a residual large enough to matter
    loss, grad = ak.ak_learned_loss_grad(*(torch.from_numpy(a).cuda() for a in (x, y, c, p)))
    want_loss, want_grad = L.loss_and_grad(p.astype(np.float64), x.astype(np.float64), y.astype(np.float64),
                                           c.astype(np.float64))
    assert loss.item() == pytest.approx(want_loss, rel=1e-3)
    g = grad.cpu().numpy().astype(np.float64)
    err = np.abs(g - want_grad) / (np.abs(want_grad) + 1e-3 * np.abs(want_grad).max())
    assert err.max() < 1e-3


def _check_all_ops(ak, keys, desc, opts):
    order = "descending" if desc else "ascending"
    p = oracle_perm(keys, desc)
    t, u = to_dev(keys)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, keys.size, ak.dtype_code(t, u), options=opts), t.device)
    ak.ak_sort(t, order, temp=temp, options=opts, unsigned=u)
    info = ak.ak_last_info(temp)
    assert info["status"] == 0
    assert_bits_equal(to_host(t, keys.dtype), oracle.gather(keys, p), "learned sort")
    t, u = to_dev(keys)
    perm = ak.ak_sortperm(t, order, options=opts, unsigned=u)
    assert np.array_equal(to_host(perm, np.uint32), p.astype(np.uint32)), "learned sortperm"
    assert_bits_equal(to_host(t, keys.dtype), keys, "sortperm keys untouched")
    vals = (np.arange(keys.size, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)).astype(np.uint32)
    t, u = to_dev(keys)
    v, _ = to_dev(vals)
    ak.ak_sort_pairs(t, v, order, options=opts, unsigned=u)
    assert_bits_equal(to_host(t, keys.dtype), oracle.gather(keys, p), "learned pair keys")
    assert_bits_equal(to_host(v, np.uint32), vals[p], "learned pair values")
    return info


@pytest.mark.parametrize("dist", synth.F64_DISTS)
@pytest.mark.parametrize("desc", [False, True])
def test_learned_six_distributions_exact(ak, dist, desc):
    """The six float64 distributions of the learned-vs-plain comparison at 2^21 keys."""
    keys = synth.dist_f64(1 << 21, dist, seed=10 + synth.F64_DISTS.index(dist))
    info = _check_all_ops(ak, keys, desc, _learned(ak))
    if dist in ("uniform", "normal", "presorted", "reversed"):
        assert info["path"] == ak.AK_PATH_LEARNED, info
    assert info["sample_size"] == (1 << 21) // 100


@pytest.mark.parametrize("dtype", [np.uint16, np.int16, np.uint32, np.int32, np.uint64, np.int64, np.float32])
def test_learned_every_dtype(ak, dtype):
    keys = synth.random_keys(300_001, dtype, seed=77, mode="bits")
    for desc in (False, True):
        _check_all_ops(ak, keys, desc, _learned(ak))


@pytest.mark.parametrize("dist,coord", [("normal", 1), ("uniform", 1), ("lognormal", 0)])
def test_model_coordinate_follows_the_sample(ak, dist, coord):
    """Float keys: the model reads the value where a normal sample is smooth
    and the radix key (log-like) where a lognormal sample's tail is; either way
    the buckets stay balanced and the output exact."""
    n = 1 << 22
    keys = synth.dist_f64(n, dist, seed=21)
    info = _check_all_ops(ak, keys, False, _learned(ak))
    assert info["path"] == ak.AK_PATH_LEARNED
    assert info["coordinate"] == coord, info
    avg = n / info["buckets"]
    assert info["max_bucket"] < 8 * avg, info


def test_adversarial_input_falls_back_exactly(ak):
    """90% of the keys share one value (one bucket far above capacity): the
    device-side check routes the call to the plain radix path."""
    n = 1 << 20
    keys = synth.normal_f32_special(n, seed=5, frac=0.001)
    keys[synth.distinct_positions(n, int(0.9 * n), seed=6)] = np.float32(1.5)
    info = _check_all_ops(ak, keys, False, _learned(ak))
    assert info["path"] == ak.AK_PATH_RADIX
    assert info["overfull_keys"] > n // 4


def test_nan_and_signed_zero_with_learned_buckets(ak):
    keys = synth.normal_f32_special(1 << 20, seed=3, frac=0.01)
    for desc in (False, True):
        _check_all_ops(ak, keys, desc, _learned(ak))


def test_mlp_residual_gain_over_piecewise_linear(ak):
    """What the trained network adds: on a heavy-tailed distribution (Pareto,
    alpha = 1.5, whose density the 64 piecewise-linear knots underfit), the
    learned path with the MLP residual trained for 64 steps puts strictly fewer
    keys in its largest bucket than the piecewise-linear CDF alone, with a
    lower training loss; both sorts stay exact."""
    n = 1 << 24
    keys = (1.0 - synth.u01_f64(44, n)) ** (-1.0 / 1.5)
    res = {}
    for steps in (-1, 64):
        opts = _learned(ak, train_steps=steps)
        t, _ = to_dev(keys)
        temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64, options=opts), t.device)
        ak.ak_sort(t, temp=temp, options=opts)
        res[steps] = ak.ak_last_info(temp)
        assert res[steps]["path"] == ak.AK_PATH_LEARNED, res[steps]
        assert_bits_equal(to_host(t, np.float64), np.sort(keys), "pareto sort")
    pl, mlp = res[-1], res[64]
    assert mlp["loss_after"] < mlp["loss_before"], mlp
    # the sample chose the residual: its largest sample bucket is strictly smaller
    assert mlp["mlp_used"] == 1 and 0 < mlp["sample_max_mlp"] < mlp["sample_max_pl"], mlp
    assert pl["mlp_used"] == 0 and pl["sample_max_mlp"] == 0 and pl["sample_max_pl"] > 0, pl
    assert mlp["max_bucket"] < pl["max_bucket"], (mlp, pl)
    assert mlp["max_bucket"] < 0.75 * pl["max_bucket"], (mlp["max_bucket"], pl["max_bucket"])


@pytest.mark.parametrize("dist", ["uniform", "normal", "lognormal"])
def test_mlp_table_choice_follows_the_sample(ak, dist):
    """The bucket table keeps the trained residual only when it strictly
    shrinks the sorted sample's largest bucket; either way the sort is exact."""
    n = 1 << 22
    keys = synth.dist_f64(n, dist, seed=10 + synth.F64_DISTS.index(dist))
    opts = _learned(ak, train_steps=32)
    t, _ = to_dev(keys)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64, options=opts), t.device)
    ak.ak_sort(t, temp=temp, options=opts)
    info = ak.ak_last_info(temp)
    assert info["path"] == ak.AK_PATH_LEARNED, info
    assert info["sample_max_pl"] > 0 and info["sample_max_mlp"] > 0, info
    assert info["mlp_used"] == (1 if info["sample_max_mlp"] < info["sample_max_pl"] else 0), info
    assert_bits_equal(to_host(t, np.float64), np.sort(keys), f"{dist} sort")


def test_auto_takes_learned_for_large_64bit_keys(ak):
    """AK_PATH_AUTO sorts 2^25+ 64-bit keys through the learned buckets (exact;
    integer keys equal under isless are bit-identical, so numpy's sort is the
    oracle's answer)."""
    n = 1 << 25
    keys = synth.uniform_i64(n, seed=8)
    t, _ = to_dev(keys)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_I64), t.device)
    ak.ak_sort(t, temp=temp)
    assert ak.ak_last_info(temp)["path"] == ak.AK_PATH_LEARNED
    assert np.array_equal(to_host(t, np.int64), np.sort(keys))
    small = synth.uniform_i64(1 << 20, seed=9)
    t, _ = to_dev(small)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT, small.size, ak.AK_I64), t.device)
    ak.ak_sort(t, temp=temp)
    assert ak.ak_last_info(temp)["path"] == ak.AK_PATH_RADIX


def test_auto_sortperm_of_64bit_keys_takes_packed_radix(ak):
    """AK_PATH_AUTO sortperm of 2^25 64-bit keys: the packed radix passes (faster
    than the learned buckets for a permutation up to 2^30 keys), exact."""
    n = 1 << 25
    keys = synth.uniform_i64(n, seed=8)
    t, _ = to_dev(keys)
    temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORTPERM, n, ak.AK_I64), t.device)
    p = ak.ak_sortperm(t, temp=temp)
    torch.cuda.synchronize()
    assert ak.ak_last_info(temp)["path"] == ak.AK_PATH_RADIX
    assert np.array_equal(to_host(p, np.uint32), oracle_perm(keys, False, threads=8).astype(np.uint32))
