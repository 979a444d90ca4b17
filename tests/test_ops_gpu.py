"""GPU parity for scans under other associative operators: running maximum
and running minimum of int32 and fp32 arrays, through the C ABI
(scan_op_i32 / scan_op_f32), every variant of single-pass, two-pass and
partitioned, against the CPU oracle.  Results are exact for both types (max
and min round nothing); fp32 inputs include NaNs, which maxNum / minNum skip,
and outputs are compared by value (so -0.0 == +0.0)."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 5119, 5120, 5121, 3 * 5120 * 7 + 13, 1_000_003]
ALGOS = ["single_pass", "two_pass", "partitioned"]


def dev():
    return torch.device("cuda", 0)


def data(key, n, seed):
    if key == "i32":
        return (synth.uniform_i32(n, 1 << 30, seed=seed) - (1 << 29)).astype(np.int32)
    f = synth.normal_f32(n, seed=seed)
    f[7::97] = np.nan
    return f


@pytest.mark.parametrize("op", ["max", "min"])
@pytest.mark.parametrize("key", ["i32", "f32"])
@pytest.mark.parametrize("algo", ALGOS)
def test_running_max_min(op, key, algo):
    dt = torch.int32 if key == "i32" else torch.float32
    kind = _capi.KIND_SCAN_MAX if op == "max" else _capi.KIND_SCAN_MIN
    for n in SIZES:
        a = data(key, n, seed=n % 1000)
        x = torch.from_numpy(a).to(dev())
        for v in range(gb.num_variants(dt, kind)):
            for excl in (False, True):
                y = gb.scan(x, excl, op=op, algo=algo, variant=v).cpu().numpy()
                assert np.array_equal(y, oracle.scan_op(a, op, excl)), (n, v, excl)
    assert gb.device_status() == 0


def test_running_max_in_place_and_abi_errors():
    n = 3 * 5120 + 5
    a = data("i32", n, seed=3)
    x = torch.from_numpy(a).to(dev())
    gb.scan(x, out=x, op="max", algo="partitioned")
    assert np.array_equal(x.cpu().numpy(), oracle.scan_op(a, "max"))
    L = _capi.lib()
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_SCAN_MAX, n))
    s = torch.cuda.current_stream().cuda_stream
    assert L.scan_op_i32(x.data_ptr(), x.data_ptr(), n, 7, 0, ws.ptr, ws.nbytes, 0, 0, s) == \
        _capi.ERR_INVALID_ARG
    assert L.scan_op_f32(x.data_ptr(), x.data_ptr(), n, 1, 0, ws.ptr, ws.nbytes, 0, 5, s) == \
        _capi.ERR_INVALID_ARG  # no such variant
    assert gb.device_status() == 0


OPS_CHUNK_SCRIPT = r"""
import sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_2312_14874_gb300 as gb
dev = torch.device("cuda", 0)
n = 16 * 5120 * 19 + 321
a = (synth.uniform_i32(n, 1 << 30, seed=5) - (1 << 29)).astype(np.int32)
f = synth.normal_f32(n, seed=6)
for arr in (a, f):
    x = torch.from_numpy(arr).to(dev)
    for op in ("max", "min"):
        for v in range(2):
            for excl in (False, True):
                y = gb.scan(x, excl, op=op, algo="partitioned", variant=v).cpu().numpy()
                assert np.array_equal(y, oracle.scan_op(arr, op, excl)), (arr.dtype, op, v, excl)
assert gb.device_status() == 0
print("ok")
"""


def test_running_max_min_partitioned_small_chunks(tmp_path):
    """The partitioned max / min scans with 16-tile chunks (child process):
    the chunk scan and the chained chunk prefixes under max and min."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    script = tmp_path / "opschunks.py"
    script.write_text(OPS_CHUNK_SCRIPT)
    env = dict(os.environ, GBSCAN_CHUNK_BYTES="4096", GBSCAN_CHUNK_LAG="2")
    r = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
