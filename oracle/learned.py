"""Float64 restatement of the learned-CDF bucketing model -- TEST INFRASTRUCTURE ONLY.

The paper's distributed sort (Sec. IV-A, SIHSort) draws a key sample, builds
"interpolated histograms" of it and turns them into splitters.  The learned path
replaces the splitters by a tiny model of the key CDF trained on that sample:

  x-hat   min-max normalised coordinate of a key, lo/hi = sample minimum/
          maximum: the order-preserving integer image of an integer key (the
          "radix key"; see ``radix_key``), the value of a float key (negated for
          a descending sort; NaN clamps to the end)
  PL(x)   64-knot piecewise-linear CDF through (xi_j, j/63), xi_j the sorted
          sample's order statistic of rank round(j (m-1) / 63): the splitters
          of the sample sort, interpolated; 0 below xi_0, 1 from xi_63 on
  r(x)    MLP residual 1 -> 16 -> 16 -> 1 with ReLU, output scaled by 1/1024
  F(x)    PL(x) + r(x), trained by mean squared error on (x_i, (i+0.5)/m) over
          the sorted sample

Correctness of the sort never depends on F: only on the bucket map being
monotone, which the tabulation enforces with a running maximum.  These functions
give the closed forms the GPU kernels are checked against: knot counts, the loss
and its gradient.  Parity of the *trained weights* is unpinned (float32 GPU
training vs this float64 restatement); they do not reach the sorted output.
"""
from __future__ import annotations

import numpy as np

N_KNOTS = 64
HIDDEN = 16
# parameter vector layout (all float): W1[16], b1[16], W2[16*16] (row-major,
# W2[j, k] multiplies h1[k] into h2[j]), b2[16], w3[16], b3[1]
P_W1, P_B1, P_W2, P_B2, P_W3, P_B3 = 0, 16, 32, 288, 304, 320
N_PARAMS = 321
OUT_SCALE = 1.0 / 1024.0  # r = OUT_SCALE * (b3 + w3 . h2)


def radix_key(keys: np.ndarray) -> np.ndarray:
    """Order-preserving map of keys to unsigned integers of the same width:
    isless(a, b) <=> radix_key(a) < radix_key(b) for non-equivalent keys, all
    NaNs map to the maximum.  Unsigned ints: identity; signed: flip the sign
    bit; floats: negative -> all bits flipped, non-negative -> sign bit flipped."""
    k = np.ascontiguousarray(keys)
    w = k.dtype.itemsize
    ut = np.dtype(f"u{w}")
    u = k.view(ut).copy()
    sign = ut.type(1 << (8 * w - 1))
    if k.dtype.kind == "u":
        return u
    if k.dtype.kind == "i":
        return u ^ sign
    neg = (u & sign) != 0
    out = np.where(neg, ~u, u ^ sign).astype(ut)
    out[np.isnan(k)] = np.iinfo(ut).max
    return out


def knot_ranks(m: int) -> np.ndarray:
    """Ranks round(j (m-1) / 63) of the 64 knots (round half up, integers)."""
    j = np.arange(N_KNOTS, dtype=np.int64)
    return (j * (m - 1) + (N_KNOTS - 1) // 2) // (N_KNOTS - 1)


def pl_knots(x_sorted: np.ndarray) -> np.ndarray:
    """The 64 knots: sample order statistics at knot_ranks (exact sample values)."""
    xs = np.asarray(x_sorted)
    return xs[knot_ranks(xs.size)]


def pl_eval(x: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Piecewise-linear interpolation through (xi_j, j/63); 0 below xi_0, 1 from
    xi_63 on.  In an interval [xi_j, xi_(j+1)) with xi_j < xi_(j+1) the value
    rises linearly from j/63 to (j+1)/63."""
    x = np.asarray(x, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.empty(x.shape)
    for i, v in enumerate(x.ravel()):
        if not v >= xi[0]:
            out.flat[i] = 0.0
        elif v >= xi[-1]:
            out.flat[i] = 1.0
        else:
            j = int(np.searchsorted(xi, v, side="right")) - 1   # xi[j] <= v < xi[j+1]
            out.flat[i] = (j + (v - xi[j]) / (xi[j + 1] - xi[j])) / (N_KNOTS - 1)
    return out


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    return (p[P_W1:P_B1], p[P_B1:P_W2], p[P_W2:P_B2].reshape(HIDDEN, HIDDEN),
            p[P_B2:P_W3], p[P_W3:P_B3], p[P_B3])


def mlp_forward(p: np.ndarray, x: np.ndarray):
    """r(x) and the activations needed by the backward pass."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    a1 = x[:, None] * W1[None, :] + b1[None, :]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2[None, :]
    h2 = np.maximum(a2, 0.0)
    r = OUT_SCALE * (h2 @ w3 + b3)
    return r, (x, a1, h1, a2, h2)


def loss_and_grad(p: np.ndarray, x: np.ndarray, y: np.ndarray, c: np.ndarray):
    """L = mean_i (PL(x_i) + r(x_i) - y_i)^2 and dL/dp (float64)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    r, (xx, a1, h1, a2, h2) = mlp_forward(p, x)
    m = xx.size
    e = pl_eval(xx, c) + r - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(e * e))
    d3 = 2.0 * e / m * OUT_SCALE           # dL/d(b3 + w3 . h2) at point i
    g = np.zeros(N_PARAMS)
    g[P_W3:P_B3] = h2.T @ d3
    g[P_B3] = d3.sum()
    d2 = (d3[:, None] * w3[None, :]) * (a2 > 0)    # dL/da2
    g[P_W2:P_B2] = (d2.T @ h1).reshape(-1)
    g[P_B2:P_W3] = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)                      # dL/da1
    g[P_W1:P_B1] = d1.T @ xx
    g[P_B1:P_W2] = d1.sum(axis=0)
    return loss, g


def adam_step(p, g, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), step counted from 1."""
    m1 = beta1 * m1 + (1 - beta1) * g
    m2 = beta2 * m2 + (1 - beta2) * g * g
    mh = m1 / (1 - beta1 ** step)
    vh = m2 / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
