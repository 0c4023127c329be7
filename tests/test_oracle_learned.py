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
    # relative error, floored at 1e-3 of the largest component (dead ReLU units
    # give exactly zero gradients)
    err = np.abs(num - g) / (np.abs(g) + np.abs(num) + 1e-3 * np.abs(g).max())
    assert err.max() < 1e-4


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences_away_from_kinks(seed):
    """The same gradient at 1e-6 relative: on points whose 32 pre-activations
    all lie at least 1e-2 from zero, a step of 1e-3 in any one parameter moves
    no pre-activation across zero (it moves one by at most 1e-3 times a weight
    or activation below 1), so the ReLU pattern is fixed.  The residual is then
    linear in each single parameter and the loss quadratic in it, and central
    differences are exact up to rounding.  Dead units: both sides exactly 0."""
    p = _params(seed)
    x = synth.u01_f64(150 + seed, 4000)
    y = np.sort(synth.u01_f64(160 + seed, 4000))
    c = np.sort(synth.u01_f64(170 + seed, L.N_KNOTS))
    _, (_, a1, _, a2, _) = L.mlp_forward(p, x)
    keep = (np.abs(a1).min(axis=1) > 1e-2) & (np.abs(a2).min(axis=1) > 1e-2)
    assert keep.sum() >= 100
    x, y = x[keep], y[keep]
    _, g = L.loss_and_grad(p, x, y, c)
    h = 1e-3
    num = np.empty_like(g)
    for i in range(L.N_PARAMS):
        e = np.zeros(L.N_PARAMS)
        e[i] = h
        num[i] = (L.loss_and_grad(p + e, x, y, c)[0] - L.loss_and_grad(p - e, x, y, c)[0]) / (2 * h)
    nz = g != 0
    assert np.all(num[~nz] == 0.0)
    assert (np.abs(num[nz] - g[nz]) / np.abs(g[nz])).max() < 1e-6


def test_zero_output_layer_reduces_to_pl_plus_bias():
    p = _params(4)
    p[L.P_W3:L.P_B3] = 0.0
    p[L.P_B3] = 0.25 / L.OUT_SCALE
    x = synth.u01_f64(5, 100)
    r, _ = L.mlp_forward(p, x)
    assert np.allclose(r, 0.25)
    c = np.linspace(0, 1, L.N_KNOTS)
    y = L.pl_eval(x, c) + 0.25
    loss, g = L.loss_and_grad(p, x, y, c)
    assert loss == pytest.approx(0.0, abs=1e-24)
    assert np.allclose(g, 0.0, atol=1e-14)


def test_pl_knots_on_uniform_sample_within_dkw_bound():
    """Dvoretzky-Kiefer-Wolfowitz: P(sup|F_m - F| > eps) <= 2 exp(-2 m eps^2); for
    the uniform CDF every sample quantile is then within eps (+1/m for the
    rank rounding) of its level.  eps = 0.005 at m = 2^20: failure < 1e-22."""
    m = 1 << 20
    xs = np.sort(synth.u01_f64(77, m).astype(np.float32))
    xi = L.pl_knots(xs).astype(np.float64)
    assert np.max(np.abs(xi - np.arange(L.N_KNOTS) / (L.N_KNOTS - 1))) < 0.005 + 1.0 / m


def test_knot_ranks_closed_form():
    # ranks round(j (m-1)/63) with halves rounded up
    assert L.knot_ranks(64).tolist() == list(range(64))
    assert L.knot_ranks(127).tolist() == [2 * j for j in range(64)]
    r = L.knot_ranks(1000)
    assert r[0] == 0 and r[-1] == 999 and np.all(np.diff(r) > 0)
    assert r[1] == 16  # 999/63 = 15.857 -> 16
    xs = np.arange(1000) / 999.0
    assert np.allclose(L.pl_knots(xs), r / 999.0)


def test_pl_interpolates_its_knots_and_is_monotone():
    xi = np.sort(synth.u01_f64(3, L.N_KNOTS))
    assert np.allclose(L.pl_eval(xi, xi), np.arange(L.N_KNOTS) / (L.N_KNOTS - 1))
    x = np.linspace(-0.5, 1.5, 4001)
    v = L.pl_eval(x, xi)
    assert np.all(np.diff(v) >= 0)
    assert v[0] == 0.0 and v[-1] == 1.0
    # uniformly spaced knots give the identity on [0, 1]
    lin = np.linspace(0, 1, L.N_KNOTS)
    xx = np.linspace(0, 1, 1001)
    assert np.allclose(L.pl_eval(xx, lin), xx)


@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.int64, np.int16, np.uint32])
def test_radix_key_orders_like_the_oracle(dtype):
    keys = synth.random_keys(20000, dtype, seed=13, mode="dups")
    by_radix = np.argsort(L.radix_key(keys), kind="stable")
    assert np.array_equal(by_radix, oracle.sortperm(keys))


def test_first_adam_step_is_signed_lr():
    g = np.array([3.0, -2.0, 1e-3])
    p, _, _ = L.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, [-0.01, 0.01, -0.01])


def test_adam_constant_gradient_moves_lr_per_step():
    """With the same gradient every step, bias correction makes m-hat = g and
    v-hat = g^2 at every step t, so each step moves -lr * sign(g): after 5
    steps p = -5 lr sign(g).  A wrong power of beta in the correction of any
    step after the first breaks this."""
    g = np.array([3.0, -2.0, 1e-3, -7.5])
    p, m1, m2 = np.zeros(4), np.zeros(4), np.zeros(4)
    for step in range(1, 6):
        p, m1, m2 = L.adam_step(p, g, m1, m2, step, lr=0.01, eps=0.0)
        assert np.allclose(p, -0.01 * step * np.sign(g), rtol=0, atol=1e-15), step


def test_adam_second_step_by_hand():
    """g1 = 1 then g2 = -1 (scalar, lr = 0.01, eps = 0): after step 1, m1 = 0.1,
    m2 = 0.001, p = -lr.  Step 2: m1 = 0.9 * 0.1 - 0.1 = -0.01, m-hat =
    -0.01 / (1 - 0.81) = -1/19; m2 = 0.999 * 0.001 + 0.001 = 0.001999, v-hat =
    0.001999 / (1 - 0.998001) = 1; p = -lr + lr / 19 = -lr * 18 / 19."""
    p, m1, m2 = L.adam_step(np.zeros(1), np.array([1.0]), np.zeros(1), np.zeros(1), 1, lr=0.01, eps=0.0)
    assert np.allclose(p, [-0.01]) and np.allclose(m1, [0.1]) and np.allclose(m2, [0.001])
    p, m1, m2 = L.adam_step(p, np.array([-1.0]), m1, m2, 2, lr=0.01, eps=0.0)
    assert np.allclose(m1, [-0.01]) and np.allclose(m2, [0.001999])
    assert np.allclose(p, [-0.01 * 18.0 / 19.0], rtol=1e-12)
