"""The no-allocation entry point, scan_inclusive_i32_noalloc.

Some callers cannot allocate device memory (code running inside a fixed-size
memory pool, an allocator callback or an accounting hook, or an embedding that
only hands over the input and output buffers).  For them the library keeps the
scan's scratch in a static device array and needs nothing but `in` and `out`.
This file checks, through the C ABI, that its results equal the CPU oracle's
element by element and those of the regular workspace-taking entry point, on
two calls in a row (the second call reuses the array the first left behind);
that sizes beyond the array's capacity and bad buffers are rejected without
touching the array; and that the stated capacity fits the array (a CPU check
of the record arithmetic).  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2312_14874_gb300 import _capi

MAX_N = 1_340_000_000
SCRATCH_BYTES = 8 << 20


def test_noalloc_capacity_fits_scratch():
    """The records of GBSCAN_NOALLOC_MAX_N elements at variant 0's tile (256 B
    header, one 8-byte word per tile plus one, in 512-byte blocks of 16 tiles)
    fit the 8 MiB array; the library checks the same at compile time."""
    import ctypes
    L = _capi.lib()
    tile = ctypes.c_int(0)
    assert L.gbscan_variant_info(_capi.I32, _capi.KIND_SCAN, 0, None, None, None,
                                 ctypes.byref(tile)) == _capi.OK
    records = (MAX_N + tile.value - 1) // tile.value + 1
    assert 256 + (records + 15) // 16 * 512 <= SCRATCH_BYTES


def reference_scan(x: torch.Tensor) -> torch.Tensor:
    """The existing entry point with its own zeroed workspace."""
    L = _capi.lib()
    n = x.numel()
    import ctypes
    size = ctypes.c_size_t(0)
    assert L.gbscan_workspace_size(_capi.I32, _capi.KIND_SCAN, n, 0, ctypes.byref(size)) == 0
    ws = torch.zeros(size.value, dtype=torch.uint8, device=x.device)
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    assert L.scan_inclusive_i32(x.data_ptr(), y.data_ptr(), n, ws.data_ptr(), size.value,
                                _capi.ALGO_SINGLE_PASS, 0, s) == _capi.OK
    return y


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_workspace_entry_point_twice():
    L = _capi.lib()
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different sizes and data: the second one runs on
    # the scratch array the first one left behind
    for call, n in enumerate((3 * 5120 * 97 + 13, (1 << 22) + 5)):
        a = synth.uniform_i32(n, 1 << 16, seed=40 + call)
        x = torch.from_numpy(a).to(dev)
        y = torch.empty_like(x)
        assert L.scan_inclusive_i32_noalloc(x.data_ptr(), y.data_ptr(), n, s) == _capi.OK
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.array_equal(got, oracle.scan_i32(a)), f"call {call}"  # integers: bit-exact
        assert torch.equal(y, reference_scan(x)), f"call {call}"


@pytest.mark.gpu
def test_noalloc_in_place_and_limits():
    L = _capi.lib()
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream().cuda_stream
    n = 100_003
    a = synth.uniform_i32(n, 256, seed=7)
    x = torch.from_numpy(a).to(dev)
    assert L.scan_inclusive_i32_noalloc(None, None, 0, s) == _capi.OK  # warm-up call
    assert L.scan_inclusive_i32_noalloc(x.data_ptr(), x.data_ptr(), n, s) == _capi.OK
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), oracle.scan_i32(a))
    # negative and over-capacity sizes, null, misaligned and partly overlapping
    # buffers are rejected before anything is launched or written
    y = torch.zeros(n + 8, dtype=torch.int32, device=dev)
    assert L.scan_inclusive_i32_noalloc(None, y.data_ptr(), n, s) == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32_noalloc(x.data_ptr(), y.data_ptr() + 2, n, s) == _capi.ERR_ALIGNMENT
    assert L.scan_inclusive_i32_noalloc(y.data_ptr(), y.data_ptr() + 4, n, s) == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32_noalloc(x.data_ptr(), x.data_ptr(), -1, s) == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32_noalloc(x.data_ptr(), x.data_ptr(), MAX_N + 1, s) == \
        _capi.ERR_UNSUPPORTED
