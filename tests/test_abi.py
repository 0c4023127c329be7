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


def test_segment_capacity_query(lib):
    """Host-only query: 80 KB of keys, values and 16-bit positions per segment,
    a multiple of 32; 0 for unsupported widths."""
    caps = {(kb, vb): lib.ak_segment_capacity(kb, vb) for kb in (2, 4, 8) for vb in (0, 1, 2, 4, 8)}
    for (kb, vb), c in caps.items():
        assert c % 32 == 0 and c == (81920 // (kb + vb + 2)) // 32 * 32, (kb, vb, c)
        assert c < 65536
    assert caps[(8, 0)] == 8192 and caps[(4, 0)] == 13632
    assert lib.ak_segment_capacity(3, 0) == 0 and lib.ak_segment_capacity(4, 3) == 0


def test_autotune_workspace_query(lib):
    """ak_autotune_temp_bytes covers every candidate plus the input copy."""
    import paper_2507_16710_gb300 as ak
    n = 1 << 20
    for op, vb in ((ak.AK_OP_SORT, 0), (ak.AK_OP_SORTPERM, 0), (ak.AK_OP_SORT_PAIRS, 4)):
        need = ak.autotune_temp_bytes(op, n, ak.AK_F64, vb)
        copy = n * (8 + (vb if op == ak.AK_OP_SORT_PAIRS else 0))
        for opts in ({"path": ak.AK_PATH_RADIX, "tile_config": 3}, {"path": ak.AK_PATH_LEARNED}):
            assert need >= ak.temp_bytes(op, n, ak.AK_F64, vb, options=opts) + copy
    out = ctypes.c_size_t(0)
    assert lib.ak_autotune_temp_bytes(ak.AK_OP_SORT_SEGMENTED, n, ak.AK_F64, 0, ctypes.byref(out)) == 1
    assert lib.ak_autotune_temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64, 0, None) == 1


def test_options_out_of_range_are_refused(lib):
    """Every documented option range is enforced at the boundary (host only)."""
    import paper_2507_16710_gb300 as ak
    out = ctypes.c_size_t(0)

    def query(**fields):
        o = ak.Options()
        for k, v in fields.items():
            setattr(o, k, v)
        return lib.ak_sort_temp_bytes(ak.AK_OP_SORT, 1 << 20, ak.AK_F64, 0, 0, ctypes.byref(o), ctypes.byref(out))

    for good in ({}, {"path": ak.AK_PATH_MERGE}, {"tile_config": 3}, {"tile_config": 4}, {"tile_config": 5}, {"bucket_bits": 8}, {"bucket_bits": 16},
                 {"train_steps": -1}, {"debug_flags": ak.AK_DEBUG_SKIP_FIRST_TILE | 2}, {"debug_flags": ak.AK_DEBUG_NO_PACK},
                 {"timeout_ns": 5},
                 {"digit_bits": 8}, {"split_caps": -1}, {"split_caps": 1}, {"split_caps": 1024}):
        assert query(**good) == 0, good
    for bad in ({"path": 5}, {"path": -1}, {"tile_config": 6}, {"tile_config": -1}, {"bucket_bits": 7}, {"bucket_bits": 17},
                {"train_steps": -2}, {"debug_flags": 8}, {"digit_bits": 11}, {"digit_bits": 4},
                {"split_caps": -2}, {"split_caps": 1025}):
        assert query(**bad) == 1, bad
    o = ak.Options()
    o.reserved[1] = 1
    assert lib.ak_sort_temp_bytes(ak.AK_OP_SORT, 10, ak.AK_U32, 0, 0, ctypes.byref(o), ctypes.byref(out)) == 1
    # malformed options are refused even by the n = 0 no-op of every entry point (no pointer touched)
    assert lib.ak_sort(None, 0, ak.AK_U32, 0, None, 0, None, ctypes.byref(o)) == 1
    assert lib.ak_sortperm(None, None, 0, ak.AK_U32, 0, None, 0, None, ctypes.byref(o)) == 1
    assert lib.ak_sort_pairs(None, None, 4, 0, ak.AK_U32, 0, None, 0, None, ctypes.byref(o)) == 1
    assert lib.ak_sort_segmented(None, None, 0, 0, ak.AK_U32, 0, None, 0, None, ctypes.byref(o)) == 1
    o.reserved[1] = 0
    assert lib.ak_sort(None, 0, ak.AK_U32, 0, None, 0, None, ctypes.byref(o)) == 0
    assert lib.ak_sort_segmented(None, None, 0, 0, ak.AK_U32, 0, None, 0, None, ctypes.byref(o)) == 0


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
    # segmented: n or nseg past 2^32 - 1 is refused before any device access
    off = ctypes.c_void_p(1 << 20)
    assert lib.ak_sort_segmented(ctypes.c_void_p(4096), off, 1, 1 << 32, ak.AK_U32, 0, None, 0, None, None) == 2
    assert lib.ak_sort_segmented(ctypes.c_void_p(4096), off, 1 << 32, 10, ak.AK_U32, 0, None, 0, None, None) == 2
    assert lib.ak_sort_segmented(ctypes.c_void_p(4096), off, -1, 10, ak.AK_U32, 0, None, 0, None, None) == 1
    # sortperm just below the UInt32 limit passes the size check (and stops at the workspace)
    assert lib.ak_sortperm(ctypes.c_void_p(4096), ctypes.c_void_p(8192), (1 << 32) - 1, ak.AK_U32, 0, None, 0,
                           None, None) == 3
    assert lib.ak_status_string(5) == b"device-side wait timed out"


def test_searchsorted_host_checks(lib):
    """Argument checks of the binary search return before any launch."""
    import paper_2507_16710_gb300 as ak
    out = ctypes.c_void_p(8192)
    x, v = ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20)
    for f in (lib.ak_searchsortedfirst, lib.ak_searchsortedlast):
        assert f(v, 10, x, 0, ak.AK_F64, 0, None, None) == 0           # m = 0: nothing to do
        assert f(None, 0, None, 0, ak.AK_F64, 0, None, None) == 0
        assert f(v, -1, x, 5, ak.AK_F64, 0, out, None) == 1            # negative n
        assert f(v, 10, x, -5, ak.AK_F64, 0, out, None) == 1           # negative m
        assert f(v, 10, x, 5, 12, 0, out, None) == 1                   # bad dtype
        assert f(v, 10, x, 5, ak.AK_F64, 2, out, None) == 1            # bad order
        assert f(v, 10, None, 5, ak.AK_F64, 0, out, None) == 1         # NULL queries
        assert f(v, 10, x, 5, ak.AK_F64, 0, None, None) == 1           # NULL output
        assert f(None, 10, x, 5, ak.AK_F64, 0, out, None) == 1         # NULL keys with n > 0
        assert f(ctypes.c_void_p(4100), 10, x, 5, ak.AK_F64, 0, out, None) == 1  # misaligned keys
        assert f(v, 10, ctypes.c_void_p(4098), 5, ak.AK_U32, 0, out, None) == 1  # misaligned queries
        assert f(v, 10, x, 5, ak.AK_U16, 0, ctypes.c_void_p(8196), None) == 1    # misaligned output


def test_accumulate_host_checks(lib):
    """Workspace query and argument checks of the scan return before any launch."""
    import paper_2507_16710_gb300 as ak
    out = ctypes.c_size_t(0)
    assert lib.ak_accumulate_temp_bytes(1 << 20, ak.AK_F32, ctypes.byref(out)) == 0
    tiles = (1 << 20) // 8192  # 32 KB tiles of float32
    assert out.value >= tiles * (4 + 8 + 8) and out.value % 256 == 0
    assert lib.ak_accumulate_temp_bytes(-1, ak.AK_F32, ctypes.byref(out)) == 1
    assert lib.ak_accumulate_temp_bytes(10, 12, ctypes.byref(out)) == 1
    for kd in (ak.AK_I128, ak.AK_U128):  # 128-bit scans are not built
        assert lib.ak_accumulate_temp_bytes(10, kd, ctypes.byref(out)) == 2
    for kd in (ak.AK_F16, ak.AK_BF16):  # valid key types the scan does not take
        assert lib.ak_accumulate_temp_bytes(10, kd, ctypes.byref(out)) == 2
    x, y, t = ctypes.c_void_p(1 << 16), ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 24)
    f = lib.ak_accumulate
    assert f(None, None, 0, ak.AK_I32, 0, 1, None, None, 0, None, None) == 0        # n = 0: nothing to do
    assert f(x, y, -1, ak.AK_I32, 0, 1, None, t, 1 << 20, None, None) == 1          # negative n
    assert f(x, y, 10, 12, 0, 1, None, t, 1 << 20, None, None) == 1                 # bad dtype
    assert f(x, y, 10, ak.AK_I128, 0, 1, None, t, 1 << 20, None, None) == 2         # unsupported
    assert f(x, y, 10, ak.AK_F16, 0, 1, None, t, 1 << 20, None, None) == 2          # unsupported
    assert f(x, y, 10, ak.AK_I32, 3, 1, None, t, 1 << 20, None, None) == 1          # bad operator
    assert f(x, y, 10, ak.AK_I32, 0, 2, None, t, 1 << 20, None, None) == 1          # bad inclusive flag
    assert f(None, y, 10, ak.AK_I32, 0, 1, None, t, 1 << 20, None, None) == 1       # NULL input
    assert f(ctypes.c_void_p((1 << 16) + 2), y, 10, ak.AK_I32, 0, 1, None, t, 1 << 20, None, None) == 1
    assert f(x, y, 10, ak.AK_I32, 0, 1, None, ctypes.c_void_p((1 << 24) + 8), 1 << 20, None, None) == 1
    assert f(x, y, 10, ak.AK_I32, 0, 1, None, None, 0, None, None) == 3             # no workspace
    assert f(x, y, 10, ak.AK_I32, 0, 1, None, t, 16, None, None) == 3               # workspace too small
    o = ak.Options()
    o.path = 9
    assert f(None, None, 0, ak.AK_I32, 0, 1, None, None, 0, None, ctypes.byref(o)) == 1  # malformed options


def test_autotune_cache_roundtrip_and_auto_sizing(lib, tmp_path):
    """The tuning cache persists as JSON lines, skips malformed lines, and an
    AK_PATH_AUTO workspace query follows a cached choice (no GPU needed)."""
    import json

    import paper_2507_16710_gb300 as ak
    lib.ak_autotune_clear()
    n = 1 << 22
    base = ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64)
    learned = ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64, options={"path": ak.AK_PATH_LEARNED})
    assert learned != base
    src = tmp_path / "in.jsonl"
    src.write_text(
        json.dumps({"op": 0, "dtype": ak.AK_F64, "log2n": 22, "val_bytes": 0, "path": ak.AK_PATH_LEARNED,
                    "tile_config": 0, "ms": 1.5}) + "\n" + "not json\n" +
        json.dumps({"op": 1, "dtype": ak.AK_U32, "log2n": 20, "val_bytes": 0, "path": 9,
                    "tile_config": 0, "ms": 1.0}) + "\n")
    ak.ak_autotune_load(str(src))
    assert ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64) == learned     # AUTO follows the cache
    assert ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64, options={"path": ak.AK_PATH_RADIX}) == base
    out = tmp_path / "out.jsonl"
    ak.ak_autotune_save(str(out))
    rows = [json.loads(x) for x in out.read_text().splitlines()]
    assert len(rows) == 1 and rows[0]["path"] == ak.AK_PATH_LEARNED and rows[0]["log2n"] == 22
    lib.ak_autotune_clear()
    assert ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64) == base
    # a tuned bucket count travels with the entry; out-of-range counts are skipped
    learned9 = ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64, options={"path": ak.AK_PATH_LEARNED, "bucket_bits": 9})
    assert learned9 != learned
    src.write_text(
        json.dumps({"op": 0, "dtype": ak.AK_F64, "log2n": 22, "val_bytes": 0, "path": ak.AK_PATH_LEARNED,
                    "tile_config": 0, "ms": 1.5, "bucket_bits": 9}) + "\n" +
        json.dumps({"op": 0, "dtype": ak.AK_F32, "log2n": 22, "val_bytes": 0, "path": ak.AK_PATH_LEARNED,
                    "tile_config": 0, "ms": 1.5, "bucket_bits": 30}) + "\n")
    ak.ak_autotune_load(str(src))
    assert ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F64) == learned9
    assert ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F32) == ak.temp_bytes(ak.AK_OP_SORT, n, ak.AK_F32,
                                                                       options={"path": ak.AK_PATH_RADIX})
    ak.ak_autotune_save(str(out))
    rows = [json.loads(x) for x in out.read_text().splitlines()]
    assert len(rows) == 1 and rows[0]["bucket_bits"] == 9
    lib.ak_autotune_clear()
    # segmented entries carry the split threshold (op 3, log2 nseg in val_bytes);
    # thresholds outside -1..1024 are skipped
    src.write_text(
        json.dumps({"op": 3, "dtype": ak.AK_U32, "log2n": 28, "val_bytes": 16, "path": ak.AK_PATH_BLOCK,
                    "tile_config": 0, "ms": 3.5, "bucket_bits": 0, "split_caps": 2}) + "\n" +
        json.dumps({"op": 3, "dtype": ak.AK_U32, "log2n": 27, "val_bytes": 16, "path": ak.AK_PATH_BLOCK,
                    "tile_config": 0, "ms": 3.5, "bucket_bits": 0, "split_caps": 5000}) + "\n")
    ak.ak_autotune_load(str(src))
    ak.ak_autotune_save(str(out))
    rows = [json.loads(x) for x in out.read_text().splitlines()]
    assert len(rows) == 1 and rows[0]["split_caps"] == 2 and rows[0]["op"] == 3
    lib.ak_autotune_clear()
    # the segmented tuner's workspace: the sort's workspace plus a copy of the keys
    got = ctypes.c_size_t(0)
    assert lib.ak_autotune_segmented_temp_bytes(1 << 20, 100, ak.AK_U32, ctypes.byref(got)) == 0
    assert got.value >= ak.temp_bytes(ak.AK_OP_SORT_SEGMENTED, 1 << 20, ak.AK_U32, nseg=100) + 4 * (1 << 20)
    assert lib.ak_autotune_segmented_temp_bytes(1 << 20, 0, ak.AK_U32, ctypes.byref(got)) == 1


def test_binding_refuses_host_tensors_and_mismatches(lib):
    """The Python binding checks its tensors before calling the library: host
    (CPU) tensors, mismatched query dtypes and wrong-sized outputs raise."""
    import torch

    import paper_2507_16710_gb300 as ak
    cpu = torch.arange(8, dtype=torch.int32)
    with pytest.raises(ValueError):
        ak.ak_sort(cpu)
    with pytest.raises(ValueError):
        ak.ak_searchsortedfirst(cpu, cpu)
    with pytest.raises(ValueError):
        ak.ak_accumulate(cpu)
    with pytest.raises(TypeError):
        ak.dtype_code(torch.zeros(2, dtype=torch.bool))
    with pytest.raises(ValueError):
        ak.order_code("sideways")
    assert ak.accumulate_temp_bytes(0, ak.AK_F64) >= 256
    with pytest.raises(ak.AkError):
        ak.accumulate_temp_bytes(-1, ak.AK_F64)


def test_sortperm_lowmem_workspace_is_smaller(lib):
    """The low-memory sortperm's workspace holds no key copy: at least 2 n x key
    bytes below ak_sortperm's radix workspace, about n x 4 bytes in all."""
    import paper_2507_16710_gb300 as ak
    n = 1 << 24
    for kd, kb in ((ak.AK_I64, 8), (ak.AK_F32, 4), (ak.AK_U16, 2), (ak.AK_BF16, 2)):
        full = ak.temp_bytes(ak.AK_OP_SORTPERM, n, kd, options={"path": ak.AK_PATH_RADIX})
        low = ak.temp_bytes(ak.AK_OP_SORTPERM_LOWMEM, n, kd)
        assert low + 2 * n * kb <= full, (kd, low, full)
        assert low < n * 4 + (n // 1000) * 1024 + (1 << 20), (kd, low)


def test_int128_host_checks(lib):
    """128-bit keys: the radix path's workspace is sized like any other key
    width; the segmented sort, the learned / block / merge paths and the
    tuner refuse them (AK_ERR_UNSUPPORTED) before any launch."""
    import paper_2507_16710_gb300 as ak
    out = ctypes.c_size_t(0)
    for kd in (ak.AK_I128, ak.AK_U128):
        for op, vb in ((ak.AK_OP_SORT, 0), (ak.AK_OP_SORTPERM, 0), (ak.AK_OP_SORT_PAIRS, 8), (ak.AK_OP_SORTPERM_LOWMEM, 0)):
            assert lib.ak_sort_temp_bytes(op, 1 << 20, kd, vb, 0, None, ctypes.byref(out)) == 0
            assert out.value > (1 << 20) * 16 or op == ak.AK_OP_SORTPERM_LOWMEM
        assert lib.ak_sort_temp_bytes(ak.AK_OP_SORT_SEGMENTED, 1 << 20, kd, 0, 4, None, ctypes.byref(out)) == 2
        for path in (ak.AK_PATH_LEARNED, ak.AK_PATH_BLOCK, ak.AK_PATH_MERGE):
            o = ak.Options()
            o.path = path
            assert lib.ak_sort_temp_bytes(ak.AK_OP_SORT, 1 << 20, kd, 0, 0, ctypes.byref(o), ctypes.byref(out)) == 2
            assert lib.ak_sort(None, 0, kd, 0, None, 0, None, ctypes.byref(o)) == 2
            assert lib.ak_sortperm(None, None, 0, kd, 0, None, 0, None, ctypes.byref(o)) == 2
        o = ak.Options()
        o.path = ak.AK_PATH_RADIX
        assert lib.ak_sort(None, 0, kd, 0, None, 0, None, ctypes.byref(o)) == 0  # n = 0 on the radix path
        assert lib.ak_sort_segmented(None, None, 0, 0, kd, 0, None, 0, None, None) == 2
        assert lib.ak_autotune_temp_bytes(ak.AK_OP_SORT, 1 << 20, kd, 0, ctypes.byref(out)) == 2
        assert lib.ak_autotune_segmented_temp_bytes(1 << 20, 4, kd, ctypes.byref(out)) == 2
    assert lib.ak_sort_temp_bytes(ak.AK_OP_SORT, 10, 12, 0, 0, None, ctypes.byref(out)) == 1  # past the last dtype


def test_int128_binding_shapes():
    """The binding reads 128-bit keys as int64 tensors of shape (n, 2)."""
    import torch
    import paper_2507_16710_gb300 as ak
    t = torch.zeros((5, 2), dtype=torch.int64)
    assert ak.key_code(t, wide=True) == (ak.AK_I128, 5)
    assert ak.key_code(t, True, wide=True) == (ak.AK_U128, 5)
    with pytest.raises(TypeError):
        ak.key_code(torch.zeros(10, dtype=torch.int64), wide=True)
    with pytest.raises(TypeError):
        ak.key_code(torch.zeros((5, 2), dtype=torch.int32), wide=True)


def test_workspace_is_the_same_for_every_tile_configuration(lib):
    """A caller sizes d_temp once; AUTO, the tuner or an explicit option may then
    pick any tile configuration (including the reduce-then-scan one with its
    chunk counts), so the radix workspace must not depend on the choice."""
    import paper_2507_16710_gb300 as ak
    for kd in (ak.AK_U16, ak.AK_F32, ak.AK_I64, ak.AK_U128):
        for op, vb in ((ak.AK_OP_SORT, 0), (ak.AK_OP_SORTPERM, 0), (ak.AK_OP_SORT_PAIRS, 4),
                       (ak.AK_OP_SORT_PAIRS, 8), (ak.AK_OP_SORTPERM_LOWMEM, 0)):
            for n in (1, 1000, 6145, 1 << 20, (1 << 30) + 7, 3 << 30):
                if op in (ak.AK_OP_SORTPERM, ak.AK_OP_SORTPERM_LOWMEM) and n >= (1 << 32):
                    continue
                sizes = {ak.temp_bytes(op, n, kd, vb, options={"path": ak.AK_PATH_RADIX, "tile_config": tc})
                         for tc in range(0, ak.AK_TILE_CONFIGS + 1)}
                assert len(sizes) == 1, (kd, op, vb, n, sizes)


def test_auto_workspace_follows_the_path_rule(lib):
    """AK_PATH_AUTO's workspace is the one of the path it will take (host
    only): sortperm of 8-byte keys up to 2^30 takes the packed radix passes,
    above that the learned buckets; the sort of 2^25+ 8-byte keys takes the
    learned buckets; 4-byte keys stay on radix."""
    import paper_2507_16710_gb300 as ak
    ak.ak_autotune_clear()
    rad = {"path": ak.AK_PATH_RADIX}
    lrn = {"path": ak.AK_PATH_LEARNED}
    for kd in (ak.AK_I64, ak.AK_F64, ak.AK_U64):
        for n in (1 << 25, 1 << 28, 1 << 30):
            # the two paths' workspaces differ, so equality names the path
            assert ak.temp_bytes(ak.AK_OP_SORTPERM, n, kd, options=rad) != \
                ak.temp_bytes(ak.AK_OP_SORTPERM, n, kd, options=lrn)
            assert ak.temp_bytes(ak.AK_OP_SORTPERM, n, kd) == ak.temp_bytes(ak.AK_OP_SORTPERM, n, kd, options=rad)
            assert ak.temp_bytes(ak.AK_OP_SORT, n, kd) == ak.temp_bytes(ak.AK_OP_SORT, n, kd, options=lrn)
        n = (1 << 30) + 7
        assert ak.temp_bytes(ak.AK_OP_SORTPERM, n, kd) == ak.temp_bytes(ak.AK_OP_SORTPERM, n, kd, options=lrn)
    for n in (1 << 25, 1 << 28):
        assert ak.temp_bytes(ak.AK_OP_SORTPERM, n, ak.AK_F32) == \
            ak.temp_bytes(ak.AK_OP_SORTPERM, n, ak.AK_F32, options=rad)
