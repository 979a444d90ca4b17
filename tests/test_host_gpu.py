"""GPU parity for the host-buffer entry point scan_inclusive_i32_host: a host
array scanned into a host array through the GPU in overlapping pieces, each
piece continuing from the ones before it (the carry kept in the workspace),
against the CPU oracle, bit-exact: pinned and pageable host memory, a
resident staging buffer and a two-slot ring, one piece and many."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n, d_elems", [(1, None), (5121, None), ((16 << 20) * 3 + 12345, None),
                                        (10_000_003, 3_000_001), (40_000_000, 16384)])
def test_host_scan(pinned, n, d_elems):
    a = synth.uniform_i32(n, 256, seed=n % 101)
    h_in = torch.from_numpy(a)
    if pinned:
        h_in = h_in.pin_memory()
    h_out = torch.empty(n, dtype=torch.int32, pin_memory=pinned)
    d_buf = None if d_elems is None else torch.empty(d_elems, dtype=torch.int32, device="cuda")
    gb.inclusive_host(h_in, h_out, d_buf=d_buf)
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy(), oracle.scan_i32(a))
    assert gb.device_status() == 0


def test_host_scan_errors():
    L = _capi.lib()
    n = 100_000
    h = torch.zeros(n, dtype=torch.int32)
    d = torch.empty(8000, dtype=torch.int32, device="cuda")
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_SCAN, n))
    s = torch.cuda.current_stream().cuda_stream
    assert L.scan_inclusive_i32_host(h.data_ptr(), h.data_ptr(), n, d.data_ptr(), 8000, ws.ptr,
                                     ws.nbytes, s) == _capi.ERR_INVALID_ARG  # ring too small
    assert L.scan_inclusive_i32_host(h.data_ptr(), h.data_ptr(), n, d.data_ptr() + 4, 4000, ws.ptr,
                                     ws.nbytes, s) == _capi.ERR_ALIGNMENT
    assert L.scan_inclusive_i32_host(None, h.data_ptr(), n, d.data_ptr(), 8000, ws.ptr, ws.nbytes, s) \
        == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32_host(None, None, 0, None, 0, ws.ptr, ws.nbytes, s) == _capi.OK
