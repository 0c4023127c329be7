"""Helpers shared by the GPU parity tests: numpy <-> torch moves and the
full-size property checks.  Expected values always come from ``oracle``."""
import numpy as np
import torch

import oracle
from oracle.learned import radix_key

_SIGNED = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32,
           np.dtype(np.uint64): np.int64}


def to_dev(a: np.ndarray):
    """numpy array -> (cuda tensor holding the same bits, unsigned flag)."""
    a = np.ascontiguousarray(a)
    if a.dtype in _SIGNED:
        return torch.from_numpy(a.view(_SIGNED[a.dtype]).copy()).cuda(), True
    return torch.from_numpy(a.copy()).cuda(), False


def to_host(t: torch.Tensor, like: np.dtype) -> np.ndarray:
    return t.cpu().numpy().view(like)


def bits(a: np.ndarray) -> np.ndarray:
    return a.view(np.dtype(f"u{a.dtype.itemsize}"))


def assert_bits_equal(got: np.ndarray, want: np.ndarray, what: str = ""):
    g, w = bits(got), bits(want)
    if g.shape != w.shape:
        raise AssertionError(f"{what}: shape {g.shape} != {w.shape}")
    bad = np.flatnonzero(g != w)
    if bad.size:
        i = int(bad[0])
        raise AssertionError(f"{what}: {bad.size} mismatches, first at {i}: got {g[i]:#x} want {w[i]:#x}")


def check_perm_properties(keys: np.ndarray, perm: np.ndarray, descending: bool):
    """A permutation p is THE stable sortperm iff (1) it is a permutation, (2) the
    keys it lists are non-decreasing in the order, (3) equivalent neighbours keep
    increasing indices.  Order is read through the oracle's radix_key, which the
    oracle tests pin against the merge-sort oracle."""
    n = keys.size
    p = perm.astype(np.int64)
    assert p.size == n
    if n == 0:
        return
    assert p.min() >= 0 and p.max() < n
    seen = np.zeros(n, dtype=bool)
    seen[p] = True
    assert seen.all(), "not a permutation"
    r = radix_key(keys)[p]
    if descending:
        r = ~r
    assert np.all(r[1:] >= r[:-1]), "not sorted"
    tie = r[1:] == r[:-1]
    assert np.all(p[1:][tie] > p[:-1][tie]), "not stable"


def oracle_perm(keys, descending, threads=1):
    return oracle.sortperm(keys, "descending" if descending else "ascending", threads=threads)
