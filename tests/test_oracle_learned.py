"""Pins for the float64 learned-CDF restatement (no GPU)."""
import numpy as np
import pytest

import oracle
from oracle import learned as L
import synth


def _params(seed):
    p = (synth.u01_f64(seed, L.N_PARAMS) - 0.5) * 0.8
    return p


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    x = synth.u01_f64(50 + seed, 257)
    y = np.sort(synth.u01_f64(60 + seed, 257))
    c = np.sort(synth.u01_f64(70 + seed, L.N_KNOTS))
    p = _params(seed)
    _, g = L.loss_and_grad(p, x, y, c)
    h = 1e-5
    num = np.empty_like(g)
    for i in range(L.N_PARAMS):
        e = np.zeros(L.N_PARAMS)
        e[i] = h
        num[i] = (L.loss_and_grad(p + e, x, y, c)[0] - L.loss_and_grad(p - e, x, y, c)[0]) / (2 * h)
    err = np.abs(num - g) / np.maximum(1e-8, np.abs(g) + np.abs(num))
    assert err.max() < 1e-6


def test_zero_output_layer_reduces_to_pl_plus_bias():
    p = _params(4)
    p[L.P_W3:L.P_B3] = 0.0
    p[L.P_B3] = 0.25
    x = synth.u01_f64(5, 100)
    r, _ = L.mlp_forward(p, x)
    assert np.allclose(r, 0.25)
    c = np.linspace(0, 1, L.N_KNOTS)
    y = L.pl_eval(x, c) + 0.25
    loss, g = L.loss_and_grad(p, x, y, c)
    assert loss == pytest.approx(0.0, abs=1e-24)
    assert np.allclose(g, 0.0, atol=1e-14)


def test_pl_knots_on_uniform_sample_within_dkw_bound():
    """Dvoretzky-Kiefer-Wolfowitz: P(sup|F_m - F| > eps) <= 2 exp(-2 m eps^2).
    eps = 0.005 at m = 2^20 gives a failure probability below 1e-22."""
    m = 1 << 20
    xs = np.sort(synth.u01_f64(77, m).astype(np.float32))
    cnt = L.pl_knot_counts(xs)
    assert cnt[0] <= 1 + 0.005 * m
    assert cnt[-1] == m
    assert np.max(np.abs(cnt / m - L.knots_u())) < 0.005


def test_pl_interpolates_its_knots_and_is_monotone():
    c = np.cumsum(synth.u01_f64(3, L.N_KNOTS))
    assert np.allclose(L.pl_eval(L.knots_u(), c), c)
    x = np.linspace(-0.5, 1.5, 10001)
    assert np.all(np.diff(L.pl_eval(x, c)) >= 0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int64, np.int16, np.uint32])
def test_radix_key_orders_like_the_oracle(dtype):
    keys = synth.random_keys(20000, dtype, seed=13, mode="dups")
    by_radix = np.argsort(L.radix_key(keys), kind="stable")
    assert np.array_equal(by_radix, oracle.sortperm(keys))


def test_first_adam_step_is_signed_lr():
    g = np.array([3.0, -2.0, 1e-3])
    p, _, _ = L.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, [-0.01, 0.01, -0.01])
