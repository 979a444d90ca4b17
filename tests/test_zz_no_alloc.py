"""The no-allocation entry point, scan_inclusive_i32_noalloc.

Some callers cannot allocate device memory (code running inside a fixed-size
memory pool, an allocator callback or an accounting hook, or an embedding that
only hands over the input and output buffers).  For them the library keeps the
scan's scratch in a static device array and needs nothing but `in` and `out`.
This file checks, through the C ABI, that its results equal those of the
regular workspace-taking entry point on two calls in a row (the second call
reuses the array the first left behind), and that sizes beyond the array's
capacity are rejected.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import synth
from paper_2312_14874_gb300 import _capi

pytestmark = pytest.mark.gpu

MAX_N = 1_340_000_000


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


def test_noalloc_matches_workspace_entry_point_twice():
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
        want = reference_scan(x)
        torch.cuda.synchronize()
        assert torch.equal(y, want), f"call {call}"  # integers: bit-exact
        assert y[-1].item() == np.int64(a.astype(np.int64).sum()).astype(np.int32)


def test_noalloc_in_place_and_limits():
    L = _capi.lib()
    dev = torch.device("cuda", 0)
    s = torch.cuda.current_stream().cuda_stream
    n = 100_003
    a = synth.uniform_i32(n, 256, seed=7)
    x = torch.from_numpy(a).to(dev)
    want = reference_scan(x)
    assert L.scan_inclusive_i32_noalloc(x.data_ptr(), x.data_ptr(), n, s) == _capi.OK
    torch.cuda.synchronize()
    assert torch.equal(x, want)
    # empty is a no-op; negative and over-capacity sizes are rejected, nothing launched
    assert L.scan_inclusive_i32_noalloc(None, None, 0, s) == _capi.OK
    assert L.scan_inclusive_i32_noalloc(x.data_ptr(), x.data_ptr(), -1, s) == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32_noalloc(x.data_ptr(), x.data_ptr(), MAX_N + 1, s) == \
        _capi.ERR_UNSUPPORTED
