"""The C-ABI library loads and exports every symbol include/ak_sort.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ak_sort.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(ak_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_16710_gb300 import _build
    _build.build()
    import paper_2507_16710_gb300 as ak
    return ak.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("ak_sort", "ak_sortperm", "ak_sort_pairs", "ak_sort_segmented",
                 "ak_sort_temp_bytes", "ak_status_check"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2507_16710_gb300 as ak
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(ak.EXPORTED)


def test_host_side_argument_checks(lib):
    import paper_2507_16710_gb300 as ak
    out = ctypes.c_size_t(0)
    assert lib.ak_sort_temp_bytes(0, -1, ak.AK_U32, 0, 0, None, ctypes.byref(out)) == 1
    assert lib.ak_sort_temp_bytes(0, 10, 99, 0, 0, None, ctypes.byref(out)) == 1
    assert lib.ak_sort_temp_bytes(2, 10, ak.AK_U32, 3, 0, None, ctypes.byref(out)) == 1
    assert lib.ak_sort_temp_bytes(0, 1 << 20, ak.AK_U32, 0, 0, None, ctypes.byref(out)) == 0
    assert out.value > 2 * 4 * (1 << 20) // 2
    # n = 0 is a no-op that touches no pointer; NULL keys with n > 0 is rejected
    assert lib.ak_sort(None, 0, ak.AK_U32, 0, None, 0, None, None) == 0
    assert lib.ak_sort(None, 5, ak.AK_U32, 0, None, 0, None, None) == 1
    assert lib.ak_sort(ctypes.c_void_p(4096), 5, ak.AK_U32, 7, None, 0, None, None) == 1
    # a workspace that is too small is refused before anything is enqueued
    assert lib.ak_sort(ctypes.c_void_p(4096), 5, ak.AK_U32, 0, ctypes.c_void_p(1 << 20), 16, None, None) == 3
    assert lib.ak_sort(ctypes.c_void_p(4096), 5, ak.AK_U32, 0, None, 0, None, None) == 3
    # misaligned workspace
    assert lib.ak_sort(ctypes.c_void_p(4096), 5, ak.AK_U32, 0, ctypes.c_void_p(4100), 1 << 30, None, None) == 1
    # UInt32 permutation limit
    assert lib.ak_sortperm(ctypes.c_void_p(4096), ctypes.c_void_p(8192), 1 << 32, ak.AK_U32, 0, None, 0,
                           None, None) == 6
    assert lib.ak_status_string(5) == b"device-side wait timed out"
