"""ctypes binding of libak_sort.so.

Argument marshalling only: every step of every sort runs in the library's CUDA
kernels.  PyTorch supplies device memory (keys, values, workspace) and the
stream.  If the compiled library is missing, every call raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("AK_SORT_LIB") or os.path.join(_HERE, "lib", "libak_sort.so")

AK_U16, AK_I16, AK_U32, AK_I32, AK_U64, AK_I64, AK_F32, AK_F64, AK_F16, AK_BF16 = range(10)
AK_I128, AK_U128 = 10, 11  # 128-bit keys: int64 tensors of shape (n, 2), [low word, high word]
AK_ASCENDING, AK_DESCENDING = 0, 1
AK_OP_SORT, AK_OP_SORTPERM, AK_OP_SORT_PAIRS, AK_OP_SORT_SEGMENTED, AK_OP_SORTPERM_LOWMEM = range(5)
AK_PATH_AUTO, AK_PATH_RADIX, AK_PATH_LEARNED, AK_PATH_BLOCK, AK_PATH_MERGE = range(5)
AK_TILE_CONFIGS = 5
AK_DEBUG_SKIP_FIRST_TILE = 1
AK_DEBUG_NO_PREFETCH = 2
AK_DEBUG_NO_PACK = 4
AK_MAX_PASSES = 16
STATUS_NAMES = {0: "AK_OK", 1: "AK_ERR_INVALID_ARG", 2: "AK_ERR_UNSUPPORTED",
                3: "AK_ERR_WORKSPACE_TOO_SMALL", 4: "AK_ERR_CUDA", 5: "AK_ERR_TIMEOUT",
                6: "AK_ERR_INDEX_OVERFLOW"}

EXPORTED = (
    "ak_sort_temp_bytes", "ak_sort", "ak_sortperm", "ak_sort_pairs", "ak_sort_segmented",
    "ak_status_check", "ak_last_info", "ak_status_string", "ak_learned_knots",
    "ak_learned_loss_grad", "ak_learned_grad_temp_bytes", "ak_autotune", "ak_autotune_save",
    "ak_autotune_load", "ak_autotune_clear", "ak_version", "ak_sort_static_scratch",
    "ak_segment_capacity", "ak_autotune_temp_bytes", "ak_searchsortedfirst", "ak_searchsortedlast",
    "ak_accumulate", "ak_accumulate_temp_bytes", "ak_sortperm_lowmem", "ak_autotune_segmented",
    "ak_autotune_segmented_temp_bytes",
)


class AkError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


class Options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("tile_config", ctypes.c_int32),
                ("bucket_bits", ctypes.c_int32), ("seed", ctypes.c_uint32),
                ("timeout_ns", ctypes.c_uint64), ("train_steps", ctypes.c_int32),
                ("debug_flags", ctypes.c_int32), ("pass_events", ctypes.c_void_p),
                ("digit_bits", ctypes.c_int32), ("split_caps", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("path", ctypes.c_int32),
                ("radix_passes", ctypes.c_int32), ("buckets", ctypes.c_int32),
                ("overfull_keys", ctypes.c_int64), ("max_bucket", ctypes.c_int64),
                ("loss_before", ctypes.c_float), ("loss_after", ctypes.c_float),
                ("sample_size", ctypes.c_int64), ("coordinate", ctypes.c_int64),
                ("mlp_used", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("sample_max_pl", ctypes.c_int64), ("sample_max_mlp", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved0"}


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libak_sort.so (build it first with __graft_entry__.build() or _build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libak_sort.so not built ({LIB_PATH}); run paper_2507_16710_gb300._build.build()")
            lib = ctypes.CDLL(LIB_PATH)
            p, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
            sz = ctypes.c_size_t
            opt = ctypes.POINTER(Options)
            sig = {
                "ak_sort_temp_bytes": ([i32, i64, i32, i32, i64, opt, ctypes.POINTER(sz)], i32),
                "ak_sort": ([p, i64, i32, i32, p, sz, p, opt], i32),
                "ak_sortperm": ([p, p, i64, i32, i32, p, sz, p, opt], i32),
                "ak_sortperm_lowmem": ([p, p, i64, i32, i32, p, sz, p, opt], i32),
                "ak_sort_pairs": ([p, p, i32, i64, i32, i32, p, sz, p, opt], i32),
                "ak_sort_segmented": ([p, p, i64, i64, i32, i32, p, sz, p, opt], i32),
                "ak_status_check": ([p, p], i32),
                "ak_last_info": ([p, p, ctypes.POINTER(Info)], i32),
                "ak_status_string": ([i32], ctypes.c_char_p),
                "ak_learned_knots": ([p, i64, p, p], i32),
                "ak_learned_loss_grad": ([p, p, i64, p, p, p, p, p, sz, p], i32),
                "ak_learned_grad_temp_bytes": ([i64], sz),
                "ak_autotune": ([i32, i64, i32, i32, i32, p, p, p, p, sz, p, opt], i32),
                "ak_autotune_save": ([ctypes.c_char_p], i32),
                "ak_autotune_load": ([ctypes.c_char_p], i32),
                "ak_autotune_clear": ([], None),
                "ak_version": ([], ctypes.c_char_p),
                "ak_sort_static_scratch": ([p, i64, i32, i32, p], i32),
                "ak_segment_capacity": ([i32, i32], i64),
                "ak_autotune_temp_bytes": ([i32, i64, i32, i32, ctypes.POINTER(sz)], i32),
                "ak_autotune_segmented": ([p, p, i64, i64, i32, i32, p, sz, p, opt], i32),
                "ak_autotune_segmented_temp_bytes": ([i64, i64, i32, ctypes.POINTER(sz)], i32),
                "ak_searchsortedfirst": ([p, i64, p, i64, i32, i32, p, p], i32),
                "ak_searchsortedlast": ([p, i64, p, i64, i32, i32, p, p], i32),
                "ak_accumulate": ([p, p, i64, i32, i32, i32, p, p, sz, p, opt], i32),
                "ak_accumulate_temp_bytes": ([i64, i32, ctypes.POINTER(sz)], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


_TORCH_DTYPE = {
    torch.int16: AK_I16, torch.int32: AK_I32, torch.int64: AK_I64,
    torch.float32: AK_F32, torch.float64: AK_F64, torch.float16: AK_F16, torch.bfloat16: AK_BF16,
}
for _name, _code in (("uint16", AK_U16), ("uint32", AK_U32), ("uint64", AK_U64)):
    if hasattr(torch, _name):
        _TORCH_DTYPE[getattr(torch, _name)] = _code


def dtype_code(t: torch.Tensor, as_unsigned: bool = False) -> int:
    """ak_dtype of a tensor; `as_unsigned` reads int16/32/64 storage as u16/32/64."""
    try:
        code = _TORCH_DTYPE[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported key dtype {t.dtype}") from None
    if as_unsigned and code in (AK_I16, AK_I32, AK_I64):
        code -= 1
    return code


def key_code(t: torch.Tensor, as_unsigned: bool = False, wide: bool = False) -> tuple[int, int]:
    """(ak_dtype, key count) of a key tensor.  `wide`: 128-bit integer keys
    held as a contiguous int64 tensor of shape (n, 2), each row the low and
    the high 64-bit word (two's complement, little-endian: the layout of
    __int128); `as_unsigned` then reads them as unsigned."""
    if not wide:
        return dtype_code(t, as_unsigned), t.numel()
    if t.dtype != torch.int64 or t.dim() != 2 or t.shape[1] != 2:
        raise TypeError("128-bit keys are an int64 tensor of shape (n, 2)")
    return (AK_U128 if as_unsigned else AK_I128), t.shape[0]


def order_code(order) -> int:
    if order in ("ascending", "asc", AK_ASCENDING, False):
        return AK_ASCENDING
    if order in ("descending", "desc", AK_DESCENDING, True):
        return AK_DESCENDING
    raise ValueError(f"bad order {order!r}")


def _check(status: int, where: str):
    if status != 0:
        raise AkError(status, where)


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _opts(options) -> ctypes.POINTER(Options) | None:
    if options is None:
        return None
    if isinstance(options, dict):
        o = Options()
        for k, v in options.items():
            if k == "pass_events":
                v = ctypes.cast(v, ctypes.c_void_p)
            setattr(o, k, v)
        options = o
    return ctypes.pointer(options)


def _contig_cuda(t: torch.Tensor, what: str):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    # the library launches on the current device with the current device's stream
    if t.device.index is not None and t.device.index != torch.cuda.current_device():
        raise ValueError(f"{what} is on {t.device}, but the current CUDA device is "
                         f"cuda:{torch.cuda.current_device()}; call under torch.cuda.device({t.device})")


def temp_bytes(op: int, n: int, kd: int, val_bytes: int = 0, nseg: int = 0, options=None) -> int:
    out = ctypes.c_size_t(0)
    _check(load().ak_sort_temp_bytes(op, n, kd, val_bytes, nseg, _opts(options), ctypes.byref(out)),
           "ak_sort_temp_bytes")
    return out.value


def workspace(nbytes: int, device) -> torch.Tensor:
    """A device workspace of nbytes (torch's allocator returns >= 512-byte alignment)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _temp_for(temp, op, n, kd, device, val_bytes=0, nseg=0, options=None):
    need = temp_bytes(op, n, kd, val_bytes, nseg, options)
    if temp is None:
        temp = workspace(need, device)
    elif temp.numel() < need:
        raise AkError(3, "workspace")
    return temp


def ak_sort(keys: torch.Tensor, order="ascending", *, temp=None, stream=None, options=None,
            unsigned: bool = False, wide: bool = False) -> torch.Tensor:
    """Stable in-place sort of a 1-D CUDA tensor (or of 128-bit keys, `wide`);
    returns `keys`."""
    _contig_cuda(keys, "keys")
    kd, n = key_code(keys, unsigned, wide)
    temp = _temp_for(temp, AK_OP_SORT, n, kd, keys.device, options=options)
    _check(load().ak_sort(keys.data_ptr(), n, kd, order_code(order), temp.data_ptr(), temp.numel(),
                          _stream_ptr(stream), _opts(options)), "ak_sort")
    return keys


def ak_sortperm(keys: torch.Tensor, order="ascending", *, perm=None, temp=None, stream=None,
                options=None, unsigned: bool = False, wide: bool = False) -> torch.Tensor:
    """Stable sorting permutation as UInt32 bits in an int32 tensor (0-based)."""
    _contig_cuda(keys, "keys")
    kd, n = key_code(keys, unsigned, wide)
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=keys.device)
    _contig_cuda(perm, "perm")
    temp = _temp_for(temp, AK_OP_SORTPERM, n, kd, keys.device, options=options)
    _check(load().ak_sortperm(keys.data_ptr(), perm.data_ptr(), n, kd, order_code(order),
                              temp.data_ptr(), temp.numel(), _stream_ptr(stream), _opts(options)),
           "ak_sortperm")
    return perm


def ak_sortperm_lowmem(keys: torch.Tensor, order="ascending", *, perm=None, temp=None, stream=None,
                       options=None, unsigned: bool = False, wide: bool = False) -> torch.Tensor:
    """ak_sortperm's permutation from a workspace without key copies (indices
    only; keys are read through them)."""
    _contig_cuda(keys, "keys")
    kd, n = key_code(keys, unsigned, wide)
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=keys.device)
    _contig_cuda(perm, "perm")
    temp = _temp_for(temp, AK_OP_SORTPERM_LOWMEM, n, kd, keys.device, options=options)
    _check(load().ak_sortperm_lowmem(keys.data_ptr(), perm.data_ptr(), n, kd, order_code(order),
                                     temp.data_ptr(), temp.numel(), _stream_ptr(stream), _opts(options)),
           "ak_sortperm_lowmem")
    return perm


def ak_sort_pairs(keys: torch.Tensor, vals: torch.Tensor, order="ascending", *, temp=None,
                  stream=None, options=None, unsigned: bool = False, wide: bool = False):
    """Stable in-place key-value sort; returns (keys, vals)."""
    _contig_cuda(keys, "keys")
    _contig_cuda(vals, "vals")
    kd, n = key_code(keys, unsigned, wide)
    if vals.numel() != n:
        raise ValueError("keys and vals differ in length")
    vb = vals.element_size()
    temp = _temp_for(temp, AK_OP_SORT_PAIRS, n, kd, keys.device, val_bytes=vb, options=options)
    _check(load().ak_sort_pairs(keys.data_ptr(), vals.data_ptr(), vb, n, kd, order_code(order),
                                temp.data_ptr(), temp.numel(), _stream_ptr(stream), _opts(options)),
           "ak_sort_pairs")
    return keys, vals


def ak_sort_segmented(keys: torch.Tensor, offsets: torch.Tensor, order="ascending", *, temp=None,
                      stream=None, options=None, unsigned: bool = False) -> torch.Tensor:
    """Sort every CSR segment keys[off[s]:off[s+1]] on its own, in place."""
    _contig_cuda(keys, "keys")
    _contig_cuda(offsets, "offsets")
    if offsets.dtype != torch.int64:
        raise TypeError("offsets must be int64")
    kd = dtype_code(keys, unsigned)
    n = keys.numel()
    nseg = offsets.numel() - 1
    temp = _temp_for(temp, AK_OP_SORT_SEGMENTED, n, kd, keys.device, nseg=nseg, options=options)
    _check(load().ak_sort_segmented(keys.data_ptr(), offsets.data_ptr(), nseg, n, kd,
                                    order_code(order), temp.data_ptr(), temp.numel(),
                                    _stream_ptr(stream), _opts(options)), "ak_sort_segmented")
    return keys


def _searchsorted(name: str, v: torch.Tensor, x: torch.Tensor, order, out, stream, unsigned: bool,
                  wide: bool = False):
    _contig_cuda(v, "v")
    _contig_cuda(x, "x")
    if x.dtype != v.dtype:
        raise TypeError(f"queries ({x.dtype}) and sorted keys ({v.dtype}) differ in dtype")
    kd, n = key_code(v, unsigned, wide)
    _, m = key_code(x, unsigned, wide)
    if out is None:
        out = torch.empty(m, dtype=torch.int64, device=x.device)
    else:
        _contig_cuda(out, "out")
        if out.dtype != torch.int64 or out.numel() != m:
            raise ValueError("out must be an int64 tensor with one element per query")
    _check(getattr(load(), name)(v.data_ptr(), n, x.data_ptr(), m, kd, order_code(order),
                                 out.data_ptr(), _stream_ptr(stream)), name)
    return out


def ak_searchsortedfirst(v: torch.Tensor, x: torch.Tensor, order="ascending", *, out=None, stream=None,
                         unsigned: bool = False, wide: bool = False) -> torch.Tensor:
    """0-based index of the first element of the sorted `v` not coming before
    each query (len(v) if none): Julia's searchsortedfirst minus one.  Fills
    `out` (int64, one per query) when given, else allocates it."""
    return _searchsorted("ak_searchsortedfirst", v, x, order, out, stream, unsigned, wide)


def ak_searchsortedlast(v: torch.Tensor, x: torch.Tensor, order="ascending", *, out=None, stream=None,
                        unsigned: bool = False, wide: bool = False) -> torch.Tensor:
    """0-based index of the last element of the sorted `v` that each query does
    not come before (-1 if none): Julia's searchsortedlast minus one."""
    return _searchsorted("ak_searchsortedlast", v, x, order, out, stream, unsigned, wide)


SCAN_OPS = {"add": 0, "max": 1, "min": 2}
_NP_DTYPE = {AK_U16: np.uint16, AK_I16: np.int16, AK_U32: np.uint32, AK_I32: np.int32,
             AK_U64: np.uint64, AK_I64: np.int64, AK_F32: np.float32, AK_F64: np.float64}


def accumulate_temp_bytes(n: int, kd: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().ak_accumulate_temp_bytes(n, kd, ctypes.byref(out)), "ak_accumulate_temp_bytes")
    return out.value


def ak_accumulate(x: torch.Tensor, op: str = "add", inclusive: bool = True, *, init=None, out=None, temp=None,
                  stream=None, options=None, unsigned: bool = False) -> torch.Tensor:
    """Prefix scan of a 1-D CUDA tensor (Sec. II-B accumulate): 'add', 'max'
    or 'min' from `init` (a host number; None = the operator's identity).
    Writes `out` when given (``out=x`` scans in place), else allocates it."""
    _contig_cuda(x, "x")
    kd = dtype_code(x, unsigned)
    if out is None:
        out = torch.empty_like(x)
    else:
        _contig_cuda(out, "out")
        if out.dtype != x.dtype or out.numel() != x.numel():
            raise ValueError("out must match x in dtype and size")
    n = x.numel()
    if temp is None:
        temp = workspace(accumulate_temp_bytes(n, kd), x.device)
    init_arr = None if init is None else np.array([init]).astype(_NP_DTYPE[kd])
    init_ptr = None if init_arr is None else init_arr.ctypes.data_as(ctypes.c_void_p)
    _check(load().ak_accumulate(x.data_ptr(), out.data_ptr(), n, kd, SCAN_OPS[op], 1 if inclusive else 0,
                                init_ptr, temp.data_ptr(), temp.numel(), _stream_ptr(stream), _opts(options)),
           "ak_accumulate")
    return out


def ak_sort_temp_bytes(op: int, n: int, kd: int, val_bytes: int = 0, nseg: int = 0, options=None) -> int:
    return temp_bytes(op, n, kd, val_bytes, nseg, options)


def ak_sort_static_scratch(keys: torch.Tensor, order="ascending", *, stream=None,
                           unsigned: bool = False) -> torch.Tensor:
    """ak_sort with the library's built-in static workspace (no allocation)."""
    _contig_cuda(keys, "keys")
    kd = dtype_code(keys, unsigned)
    _check(load().ak_sort_static_scratch(keys.data_ptr(), keys.numel(), kd, order_code(order),
                                         _stream_ptr(stream)), "ak_sort_static_scratch")
    return keys


def ak_status_check(temp: torch.Tensor, stream=None) -> int:
    return load().ak_status_check(temp.data_ptr(), _stream_ptr(stream))


def ak_last_info(temp: torch.Tensor, stream=None) -> dict:
    info = Info()
    _check(load().ak_last_info(temp.data_ptr(), _stream_ptr(stream), ctypes.byref(info)), "ak_last_info")
    return info.as_dict()


def ak_status_string(status: int) -> str:
    return load().ak_status_string(status).decode()


def ak_version() -> str:
    return load().ak_version().decode()


def ak_segment_capacity(key_bytes: int, val_bytes: int = 0) -> int:
    """Keys of one segment sorted in shared memory (see include/ak_sort.h)."""
    return int(load().ak_segment_capacity(key_bytes, val_bytes))


def ak_learned_knots(xs_sorted: torch.Tensor, stream=None) -> torch.Tensor:
    _contig_cuda(xs_sorted, "xs")
    knots = torch.empty(64, dtype=torch.float32, device=xs_sorted.device)
    _check(load().ak_learned_knots(xs_sorted.data_ptr(), xs_sorted.numel(), knots.data_ptr(),
                                   _stream_ptr(stream)), "ak_learned_knots")
    return knots


def ak_learned_loss_grad(x: torch.Tensor, y: torch.Tensor, c: torch.Tensor, params: torch.Tensor,
                         stream=None):
    for t, w in ((x, "x"), (y, "y"), (c, "c"), (params, "params")):
        _contig_cuda(t, w)
    m = x.numel()
    grad = torch.empty(321, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    temp = workspace(load().ak_learned_grad_temp_bytes(m), x.device)
    _check(load().ak_learned_loss_grad(x.data_ptr(), y.data_ptr(), m, c.data_ptr(), params.data_ptr(),
                                       grad.data_ptr(), loss.data_ptr(), temp.data_ptr(), temp.numel(),
                                       _stream_ptr(stream)), "ak_learned_loss_grad")
    return loss, grad


def autotune_temp_bytes(op: int, n: int, kd: int, val_bytes: int = 0) -> int:
    """Workspace ak_autotune needs: the largest candidate plus a copy of the inputs."""
    out = ctypes.c_size_t(0)
    _check(load().ak_autotune_temp_bytes(op, n, kd, val_bytes, ctypes.byref(out)), "ak_autotune_temp_bytes")
    return out.value


def ak_autotune(op: int, keys: torch.Tensor, order="ascending", vals=None, perm=None, temp=None,
                stream=None, unsigned: bool = False) -> Options:
    """Time the candidates for this call shape and cache the fastest; returns it."""
    kd = dtype_code(keys, unsigned)
    n = keys.numel()
    vb = vals.element_size() if vals is not None else 0
    if temp is None:
        temp = workspace(autotune_temp_bytes(op, n, kd, vb), keys.device)
    best = Options()
    _check(load().ak_autotune(op, n, kd, vb, order_code(order), keys.data_ptr(),
                              vals.data_ptr() if vals is not None else None,
                              perm.data_ptr() if perm is not None else None, temp.data_ptr(),
                              temp.numel(), _stream_ptr(stream), ctypes.byref(best)), "ak_autotune")
    return best


def ak_autotune_segmented(keys: torch.Tensor, offsets: torch.Tensor, order="ascending", temp=None, stream=None,
                          unsigned: bool = False) -> Options:
    """Time the split thresholds of ak_sort_segmented on this batch and cache
    the fastest; returns it (split_caps)."""
    _contig_cuda(keys, "keys")
    _contig_cuda(offsets, "offsets")
    kd = dtype_code(keys, unsigned)
    n, nseg = keys.numel(), offsets.numel() - 1
    if temp is None:
        out = ctypes.c_size_t(0)
        _check(load().ak_autotune_segmented_temp_bytes(n, nseg, kd, ctypes.byref(out)),
               "ak_autotune_segmented_temp_bytes")
        temp = workspace(out.value, keys.device)
    best = Options()
    _check(load().ak_autotune_segmented(keys.data_ptr(), offsets.data_ptr(), nseg, n, kd, order_code(order),
                                        temp.data_ptr(), temp.numel(), _stream_ptr(stream), ctypes.byref(best)),
           "ak_autotune_segmented")
    return best


def ak_autotune_save(path: str):
    _check(load().ak_autotune_save(path.encode()), "ak_autotune_save")


def ak_autotune_load(path: str):
    _check(load().ak_autotune_load(path.encode()), "ak_autotune_load")


def ak_autotune_clear():
    load().ak_autotune_clear()
