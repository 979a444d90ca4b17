"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; host-side argument checks run without a GPU (they return
before any CUDA call)."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT

import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*"
                             r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("scan_inclusive_i32", "scan_exclusive_i32", "scan_inclusive_i64",
                 "scan_exclusive_i64", "scan_inclusive_f32", "scan_exclusive_f32",
                 "scan_segmented_batched_i32", "scan_segmented_batched_f32",
                 "scan_backward_f32", "scan_get_device_status", "gbscan_workspace_size",
                 "gbscan_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = _capi.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _capi.exported_names(), f"{name} has no binding"
    assert lib.gbscan_abi_version() == _capi.ABI_VERSION


def test_workspace_size():
    out = ctypes.c_size_t(0)
    L = _capi.lib()
    assert L.gbscan_workspace_size(_capi.I32, _capi.KIND_SCAN, 1 << 30, 0, ctypes.byref(out)) == 0
    # header + 512-byte blocks of 16 tile records, one record per smallest
    # tile (3072 elements) plus one
    records = -(-(1 << 30) // 3072) + 1
    assert out.value == 256 + 512 * (-(-records // 16))
    # segmented calls add the head bitmap: one bit per element plus 16384
    # elements of padding, in 16-byte units
    n = 386099019
    assert L.gbscan_workspace_size(_capi.I32, _capi.KIND_SEGMENTED, n, 65536, ctypes.byref(out)) == 0
    records = -(-n // 3072) + 1
    assert out.value == 256 + 512 * (-(-records // 16)) + 16 * ((n + 16384 + 127) // 128)
    assert L.gbscan_workspace_size(_capi.I32, _capi.KIND_SCAN, -1, 0, ctypes.byref(out)) == \
        _capi.ERR_INVALID_ARG
    assert L.gbscan_workspace_size(9, _capi.KIND_SCAN, 10, 0, ctypes.byref(out)) == \
        _capi.ERR_INVALID_ARG
    assert L.gbscan_workspace_size(_capi.I32, _capi.KIND_SCAN, 10, 0, None) == \
        _capi.ERR_INVALID_ARG
    assert L.gbscan_workspace_size(_capi.I32, _capi.KIND_SCAN, 1 << 50, 0,
                                   ctypes.byref(out)) == _capi.ERR_UNSUPPORTED


def test_host_argument_errors_without_gpu():
    """Every check below fails before any CUDA call, so it runs on CPU."""
    L = _capi.lib()
    fake = 1 << 40  # never dereferenced
    ws = 1 << 41
    # negative n, bad algo, bad variant
    assert L.scan_inclusive_i32(fake, fake, -1, ws, 1 << 20, 0, 0, None) == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32(fake, fake, 10, ws, 1 << 20, 7, 0, None) == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32(fake, fake, 10, ws, 1 << 20, 0, 99, None) == _capi.ERR_INVALID_ARG
    # n == 0 is a no-op even with null pointers
    assert L.scan_inclusive_i32(None, None, 0, None, 0, 0, 0, None) == _capi.OK
    # null pointers
    assert L.scan_inclusive_i32(None, fake, 10, ws, 1 << 20, 0, 0, None) == _capi.ERR_INVALID_ARG
    # misaligned to the element size
    assert L.scan_inclusive_i64(fake + 4, fake + (1 << 20), 10, ws, 1 << 20, 0, 0, None) == \
        _capi.ERR_ALIGNMENT
    # partial overlap
    assert L.scan_inclusive_i32(fake, fake + 8, 10, ws, 1 << 20, 0, 0, None) == \
        _capi.ERR_INVALID_ARG
    # workspace: null, misaligned, too small
    assert L.scan_inclusive_i32(fake, fake, 10, None, 1 << 20, 0, 0, None) == _capi.ERR_WORKSPACE
    assert L.scan_inclusive_i32(fake, fake, 10, ws + 8, 1 << 20, 0, 0, None) == _capi.ERR_WORKSPACE
    assert L.scan_inclusive_i32(fake, fake, 1 << 20, ws, 1024, 0, 0, None) == _capi.ERR_WORKSPACE
    # f32 bad mode
    assert L.scan_inclusive_f32(fake, fake, 10, 5, ws, 1 << 20, 0, 0, None) == \
        _capi.ERR_INVALID_ARG
    # segmented: no segments for a nonempty array, misaligned offsets
    assert L.scan_segmented_batched_i32(fake, fake, 10, fake, 0, 0, ws, 1 << 20, 0, None) == \
        _capi.ERR_INVALID_ARG
    assert L.scan_segmented_batched_i32(fake, fake, 10, fake + 4, 2, 0, ws, 1 << 20, 0, None) == \
        _capi.ERR_ALIGNMENT
    # rows: negative sizes; empty is a no-op
    assert L.scan_rows_f32(fake, fake, -1, 4, 0, ws, 1 << 20, 0, None) == _capi.ERR_INVALID_ARG
    assert L.scan_backward_f32(None, None, 0, 4, 0, None, 0, 0, None) == _capi.OK
    # copy: overlap and misalignment
    assert L.gbscan_copy(fake, fake + 16, 64, None) == _capi.ERR_INVALID_ARG
    assert L.gbscan_copy(fake, fake + 4096, 60, None) == _capi.ERR_ALIGNMENT


def test_variant_table():
    L = _capi.lib()
    for dt in (_capi.I32, _capi.I64, _capi.F32, _capi.F64):
        nv = L.gbscan_num_variants(dt, _capi.KIND_SCAN)
        assert nv >= 1
        t, i, s, tile = (ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int())
        for v in range(nv):
            assert L.gbscan_variant_info(dt, _capi.KIND_SCAN, v, ctypes.byref(t), ctypes.byref(i),
                                         ctypes.byref(s), ctypes.byref(tile)) == 0
            # threads counts the loader warp and one agent warp per stage
            assert tile.value == (t.value - 32 * (1 + s.value)) * i.value
            esz = 8 if dt in (_capi.I64, _capi.F64) else 4
            assert (i.value * esz) % 16 == 0
            assert ((i.value * esz) // 16) % 2 == 1  # odd vectors: conflict-free LDS.128
    assert L.gbscan_num_variants(_capi.I64, _capi.KIND_SEGMENTED) == 0


def test_compaction_variant_table():
    """Compaction variants 0-2 are the partitioned kernel (consumer warps plus a
    loader and a scanner warp), variant 3 the single-pass one (consumer warps
    plus a loader and one agent warp per stage); every tile is whole rows of
    16-byte flag vectors (bulk copies of the flags, the agents' row reads)
    and no smaller than the tile the workspace size assumes."""
    L = _capi.lib()
    for dt in (_capi.I32, _capi.F32):
        assert L.gbscan_num_variants(dt, _capi.KIND_COMPACT) == 4
        t, i, s, tile = (ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int())
        for v in range(4):
            assert L.gbscan_variant_info(dt, _capi.KIND_COMPACT, v, ctypes.byref(t), ctypes.byref(i),
                                         ctypes.byref(s), ctypes.byref(tile)) == 0
            helpers = 32 * 2 if v < 3 else 32 * (1 + s.value)
            assert tile.value == (t.value - helpers) * i.value, v
            assert tile.value % (16 * 32) == 0 and tile.value >= 256 * 12, v
            assert i.value % 4 == 0, v
    assert L.gbscan_num_variants(_capi.I64, _capi.KIND_COMPACT) == 0


def test_resident_max_n_arguments():
    L = _capi.lib()
    n = ctypes.c_int64(0)
    assert L.gbscan_resident_max_n(_capi.I32, _capi.KIND_SCAN, 0, None) == _capi.ERR_INVALID_ARG
    assert L.gbscan_resident_max_n(99, _capi.KIND_SCAN, 0, ctypes.byref(n)) == _capi.ERR_INVALID_ARG
    assert L.gbscan_resident_max_n(_capi.F32, _capi.KIND_SCAN, 7, ctypes.byref(n)) == _capi.ERR_INVALID_ARG
    for kind in (_capi.KIND_ROWS, _capi.KIND_SEGMENTED, _capi.KIND_COMPACT):
        assert L.gbscan_resident_max_n(_capi.F32, kind, 0, ctypes.byref(n)) == _capi.ERR_UNSUPPORTED
    assert L.gbscan_resident_max_n(_capi.F64, _capi.KIND_SCAN_MAX, 0, ctypes.byref(n)) == \
        _capi.ERR_UNSUPPORTED


def test_status_strings():
    L = _capi.lib()
    for code in range(7):
        assert L.gbscan_status_string(code)
    assert L.gbscan_status_string(99) == b"unknown status"


def test_cpu_tensors_are_rejected():
    import torch
    with pytest.raises(TypeError):
        gb.inclusive(torch.arange(10, dtype=torch.int32))
