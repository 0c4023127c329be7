"""CPU oracle for the single-device sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this package.  It shares no code with the CUDA library, and the library
never calls it.

``ak_oracle.c`` is a plain top-down stable merge sort under Julia ``isless`` (the
sort, sortperm and by-key sort of Sec. II-B, used as the rank-local sort of the
sample sort in Sec. IV-A), and a textbook bisection for the binary searches of
Sec. II-B (searchsortedfirst / searchsortedlast) and a left-to-right prefix scan
for its accumulate.  ``learned.py`` restates the learned-CDF model in
float64 numpy.  This module compiles the C file with gcc on first use and wraps
it with ctypes over numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ak_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# dtype codes of ak_oracle.c
_DTYPE_CODE = {
    np.dtype(np.uint16): 0, np.dtype(np.int16): 1, np.dtype(np.uint32): 2,
    np.dtype(np.int32): 3, np.dtype(np.uint64): 4, np.dtype(np.int64): 5,
    np.dtype(np.float32): 6, np.dtype(np.float64): 7, np.dtype(np.float16): 8,
}
BF16_CODE = 9  # bfloat16 keys travel as their uint16 bits: pass as_dtype="bfloat16"
# 128-bit integer keys travel as 16-byte void elements (np.dtype("V16"), low 8
# bytes first): pass as_dtype="int128" or "uint128"
I128_CODES = {"int128": 10, "uint128": 11}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (portable C, no -march flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            lib.oracle_sortperm.argtypes = [p, i64, i32, i32, p]
            lib.oracle_sortperm_threaded.argtypes = [p, i64, i32, i32, p, i32]
            lib.oracle_sortperm_segmented.argtypes = [p, p, i64, i64, i32, i32, p]
            lib.oracle_gather.argtypes = [p, p, i64, i32, p]
            lib.oracle_isless_pairs.argtypes = [p, p, i64, i32, p]
            lib.oracle_searchsorted.argtypes = [p, i64, p, i64, i32, i32, i32, p]
            lib.oracle_accumulate.argtypes = [p, i64, i32, i32, i32, p, p]
            for f in (lib.oracle_sortperm, lib.oracle_sortperm_threaded,
                      lib.oracle_sortperm_segmented, lib.oracle_gather,
                      lib.oracle_isless_pairs, lib.oracle_searchsorted, lib.oracle_accumulate):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _code(a: np.ndarray, as_dtype=None) -> int:
    if as_dtype == "bfloat16":
        if a.dtype != np.uint16:
            raise TypeError("bfloat16 keys are passed as their uint16 bits")
        return BF16_CODE
    if as_dtype in I128_CODES:
        if a.dtype.itemsize != 16 or a.dtype.kind != "V":
            raise TypeError("128-bit keys are passed as 16-byte void elements (np.dtype('V16'))")
        return I128_CODES[as_dtype]
    if as_dtype is not None:
        raise ValueError(as_dtype)
    try:
        return _DTYPE_CODE[a.dtype]
    except KeyError:
        raise TypeError(f"oracle: unsupported key dtype {a.dtype}") from None


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _desc(order) -> int:
    if order in ("ascending", "asc", 0, False):
        return 0
    if order in ("descending", "desc", 1, True):
        return 1
    raise ValueError(order)


def sortperm(keys: np.ndarray, order="ascending", threads: int = 1, as_dtype=None) -> np.ndarray:
    """Stable sorting permutation (int64, 0-based)."""
    k = np.ascontiguousarray(keys)
    perm = np.empty(k.size, dtype=np.int64)
    lib = _load()
    if threads > 1:
        rc = lib.oracle_sortperm_threaded(_ptr(k), k.size, _code(k, as_dtype), _desc(order), _ptr(perm), threads)
    else:
        rc = lib.oracle_sortperm(_ptr(k), k.size, _code(k, as_dtype), _desc(order), _ptr(perm))
    if rc:
        raise RuntimeError(f"oracle_sortperm failed ({rc})")
    return perm


def gather(src: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """src[perm], moving raw bits."""
    s = np.ascontiguousarray(src)
    p = np.ascontiguousarray(perm, dtype=np.int64)
    out = np.empty(p.size, dtype=s.dtype)
    if _load().oracle_gather(_ptr(s), _ptr(p), p.size, s.dtype.itemsize, _ptr(out)):
        raise RuntimeError("oracle_gather failed")
    return out


def sort(keys: np.ndarray, order="ascending", threads: int = 1, as_dtype=None) -> np.ndarray:
    return gather(keys, sortperm(keys, order, threads, as_dtype))


def sort_pairs(keys: np.ndarray, vals: np.ndarray, order="ascending", threads: int = 1, as_dtype=None):
    p = sortperm(keys, order, threads, as_dtype)
    return gather(keys, p), gather(vals, p)


def sortperm_segmented(keys: np.ndarray, offsets: np.ndarray, order="ascending", as_dtype=None) -> np.ndarray:
    """Global-index permutation sorting each CSR segment on its own."""
    k = np.ascontiguousarray(keys)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    perm = np.empty(k.size, dtype=np.int64)
    rc = _load().oracle_sortperm_segmented(_ptr(k), _ptr(off), off.size - 1, k.size, _code(k, as_dtype),
                                           _desc(order), _ptr(perm))
    if rc:
        raise RuntimeError(f"oracle_sortperm_segmented failed ({rc})")
    return perm


def sort_segmented(keys: np.ndarray, offsets: np.ndarray, order="ascending", as_dtype=None) -> np.ndarray:
    return gather(keys, sortperm_segmented(keys, offsets, order, as_dtype))


def isless(a: np.ndarray, b: np.ndarray, as_dtype=None) -> np.ndarray:
    """Elementwise Julia isless(a[i], b[i]) as computed by the oracle."""
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b, dtype=a.dtype)
    out = np.empty(a.size, dtype=np.uint8)
    if _load().oracle_isless_pairs(_ptr(a), _ptr(b), a.size, _code(a, as_dtype), _ptr(out)):
        raise RuntimeError("oracle_isless_pairs failed")
    return out.astype(bool)


def searchsorted(v: np.ndarray, x: np.ndarray, side: str = "first", order="ascending", as_dtype=None) -> np.ndarray:
    """Binary search of Sec. II-B over a v already in the order's sequence.

    side 'first': index of the first v element not coming before x (n if none);
    side 'last' : index of the last v element x does not come before (-1 if none).
    Both 0-based (Julia's searchsortedfirst / searchsortedlast minus one), int64.
    """
    vv = np.ascontiguousarray(v)
    xx = np.ascontiguousarray(x, dtype=vv.dtype)
    if side not in ("first", "last"):
        raise ValueError(side)
    out = np.empty(xx.size, dtype=np.int64)
    rc = _load().oracle_searchsorted(_ptr(vv), vv.size, _ptr(xx), xx.size, _code(vv, as_dtype), _desc(order),
                                     0 if side == "first" else 1, _ptr(out))
    if rc:
        raise RuntimeError(f"oracle_searchsorted failed ({rc})")
    return out


ACCUMULATE_OPS = {"add": 0, "max": 1, "min": 2}


def accumulate(x: np.ndarray, op: str = "add", inclusive: bool = True, init=None) -> np.ndarray:
    """Prefix scan of Sec. II-B (accumulate), left to right from ``init``.

    inclusive: out[i] = init op x[0] op ... op x[i]; exclusive: the same up to
    x[i-1] (out[0] = init).  op 'add' wraps for integers and is a compensated
    float64 sum rounded once per output for floats; 'max' / 'min' are Julia's
    (NaN wins, -0.0 below +0.0).  ``init`` defaults to the op's identity.
    """
    xx = np.ascontiguousarray(x)
    code = ACCUMULATE_OPS[op]
    if init is None:
        init = identity(xx.dtype, op)
    iv = np.array([init], dtype=xx.dtype)
    out = np.empty_like(xx)
    rc = _load().oracle_accumulate(_ptr(xx), xx.size, _code(xx), code, 1 if inclusive else 0, _ptr(iv), _ptr(out))
    if rc:
        raise RuntimeError(f"oracle_accumulate failed ({rc})")
    return out


def identity(dtype, op: str):
    """The start value that changes nothing, bit for bit: 0 for integer add
    and -0.0 for float add (x + -0.0 is x, -0.0 included); the dtype's lowest
    (max) or highest (min) value, -Inf / +Inf for floats."""
    dt = np.dtype(dtype)
    if op == "add":
        return dt.type(-0.0) if dt.kind == "f" else dt.type(0)
    if dt.kind == "f":
        return dt.type(-np.inf if op == "max" else np.inf)
    info = np.iinfo(dt)
    return dt.type(info.min if op == "max" else info.max)


def _word_bits(v) -> np.ndarray:
    """64-bit words as uint64 bits: integer arrays by two's complement, other
    sequences element by element as Python ints (either sign)."""
    if isinstance(v, np.ndarray) and v.dtype.kind in "iu":
        return v.astype(np.uint64)
    return np.array([int(t) & 0xFFFFFFFFFFFFFFFF for t in v], dtype=np.uint64)


def int128_from_words(lo, hi) -> np.ndarray:
    """128-bit keys (V16 elements) from their low and high 64-bit words."""
    lo, hi = _word_bits(lo), _word_bits(hi)
    w = np.empty((lo.size, 2), dtype=np.uint64)
    w[:, 0] = lo
    w[:, 1] = hi
    return w.view(np.dtype("V16")).reshape(-1)


def int128_words(keys: np.ndarray):
    """(low, high) uint64 words of V16 keys."""
    w = np.ascontiguousarray(keys).view(np.uint64).reshape(-1, 2)
    return w[:, 0].copy(), w[:, 1].copy()
