"""GPU parity for scans under other associative operators and dtypes: running
maximum and minimum of int32, int64, uint32 and fp32 arrays (scan_op_*),
uint32 sums (scan_{inclusive,exclusive}_u32), and segmented running maximum
and minimum (scan_segmented_op_*), every variant of every algorithm, through
the C ABI, against the CPU oracle.  Results are exact for both types (max
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
ALGOS = ["single_pass", "two_pass", "partitioned", "resident"]


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


# ---- uint32 sums, int64 and uint32 maxima / minima ------------------------------

def u32_data(n, seed):
    """Every uint32 value is possible, including those with the top bit set,
    whose unsigned order differs from the signed order of the same bits."""
    return synth.uniform_i64(n, 1 << 32, seed=seed).astype(np.uint32)


def i64_data(n, seed):
    return synth.uniform_i64(n, 1 << 32, seed=seed).astype(np.int64) * 1_000_003 - (1 << 50)


def to_dev_u32(a):
    return torch.from_numpy(a.view(np.int32)).to(dev()).view(torch.uint32)


@pytest.mark.parametrize("algo", ALGOS)
def test_uint32_sums(algo):
    """uint32 sums (modulo 2^32) through the C ABI against the unsigned oracle,
    bit-exact, every variant, inclusive and exclusive."""
    L = _capi.lib()
    s = torch.cuda.current_stream().cuda_stream
    a_ = gb._ALGOS[algo]
    for n in SIZES:
        a = u32_data(n, seed=n % 1000)
        x = to_dev_u32(a)
        y = torch.empty_like(x)
        ws = gb.Workspace(gb.workspace_bytes(torch.uint32, _capi.KIND_SCAN, n))
        for v in range(gb.num_variants(torch.uint32)):
            for excl in (False, True):
                fn = L.scan_exclusive_u32 if excl else L.scan_inclusive_u32
                assert fn(x.data_ptr(), y.data_ptr(), n, ws.ptr, ws.nbytes, a_, v, s) == _capi.OK
                got = y.view(torch.int32).cpu().numpy().view(np.uint32)
                assert np.array_equal(got, oracle.scan_u32(a, excl)), (n, v, excl)
        assert gb.device_status(ws) == 0


@pytest.mark.parametrize("op", ["max", "min"])
@pytest.mark.parametrize("key", ["i64", "u32"])
@pytest.mark.parametrize("algo", ALGOS)
def test_running_max_min_int64_uint32(op, key, algo):
    dt = torch.int64 if key == "i64" else torch.uint32
    kind = _capi.KIND_SCAN_MAX if op == "max" else _capi.KIND_SCAN_MIN
    for n in SIZES:
        a = i64_data(n, seed=n % 1000) if key == "i64" else u32_data(n, seed=n % 1000)
        x = torch.from_numpy(a).to(dev()) if key == "i64" else to_dev_u32(a)
        for v in range(gb.num_variants(dt, kind)):
            for excl in (False, True):
                y = gb.scan(x, excl, op=op, algo=algo, variant=v)
                got = y.cpu().numpy() if key == "i64" else y.view(torch.int32).cpu().numpy().view(np.uint32)
                assert np.array_equal(got, oracle.scan_op(a, op, excl)), (n, v, excl)
    assert gb.device_status() == 0


# ---- segmented maxima / minima --------------------------------------------------

def seg_offsets(n_seg, seed, max_len):
    """CSR offsets with about a fifth of the segments empty."""
    lens = synth.uniform_i64(n_seg, max_len + 1, seed=seed, stream=1)
    lens = np.where(synth.unit_f32(n_seg, seed=seed, stream=2) < 0.2, 0, lens)
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


@pytest.mark.parametrize("op", ["max", "min"])
@pytest.mark.parametrize("key", ["i32", "f32"])
def test_segmented_max_min(op, key):
    """Segmented running maximum / minimum (every segment restarts; exclusive
    segments start from the identity), short and long segments, empty ones,
    fp32 with NaNs, every variant, against the oracle, exact."""
    dt = torch.int32 if key == "i32" else torch.float32
    kind = _capi.KIND_SEGMENTED_MAX if op == "max" else _capi.KIND_SEGMENTED_MIN
    for n_seg, max_len, seed in ((1, 7000, 1), (37, 40, 2), (500, 3000, 3), (3000, 900, 4)):
        off = seg_offsets(n_seg, seed, max_len)
        n = int(off[-1])
        if n == 0:
            continue
        a = data(key, n, seed=seed)
        if key == "f32":
            a[off[:-1][off[:-1] < n][::3]] = np.nan  # NaN segment heads: skipped, as maxNum does
        x = torch.from_numpy(a).to(dev())
        o = torch.from_numpy(off).to(dev())
        for v in range(gb.num_variants(dt, kind)):
            for excl in (False, True):
                y = gb.segmented(x, o, excl, op=op, variant=v).cpu().numpy()
                assert np.array_equal(y, oracle.seg_scan_op(a, off, op, excl)), (n_seg, v, excl)
    assert gb.device_status() == 0


def test_segmented_op_abi_errors():
    L = _capi.lib()
    n = 100
    x = torch.zeros(n, dtype=torch.int32, device=dev())
    o = torch.tensor([0, 40, n], dtype=torch.int64, device=dev())
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_SEGMENTED_MAX, n, 2))
    s = torch.cuda.current_stream().cuda_stream
    assert L.scan_segmented_op_i32(x.data_ptr(), x.data_ptr(), n, o.data_ptr(), 2, 9, 0, ws.ptr,
                                   ws.nbytes, 0, s) == _capi.ERR_INVALID_ARG  # no such op
    assert L.scan_segmented_op_f32(x.data_ptr(), x.data_ptr(), n, o.data_ptr(), 2, 1, 0, ws.ptr,
                                   ws.nbytes, 7, s) == _capi.ERR_INVALID_ARG  # no such variant
    assert L.scan_op_u32(x.data_ptr(), x.data_ptr(), n, 5, 0, ws.ptr, ws.nbytes, 0, 0, s) == \
        _capi.ERR_INVALID_ARG
    assert gb.device_status(ws) == 0


SEG_OPS_CHUNK_SCRIPT = r"""
import sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_2312_14874_gb300 as gb
dev = torch.device("cuda", 0)
off = synth.segment_offsets(300, max_log2=12, seed=3)
n = int(off[-1])
o = torch.from_numpy(off).to(dev)
a = (synth.uniform_i32(n, 1 << 30, seed=5) - (1 << 29)).astype(np.int32)
f = synth.normal_f32(n, seed=6)
for arr in (a, f):
    x = torch.from_numpy(arr).to(dev)
    for op in ("max", "min"):
        for v in range(2):
            for excl in (False, True):
                y = gb.segmented(x, o, excl, op=op, variant=v).cpu().numpy()
                assert np.array_equal(y, oracle.seg_scan_op(arr, off, op, excl)), (arr.dtype, op, v, excl)
assert gb.device_status() == 0
print("ok")
"""


def test_segmented_max_min_small_chunks(tmp_path):
    """Segmented max / min with 16-tile chunks (child process): the chunk scan
    of (head, value) pairs and the chained chunk prefixes under max and min."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    script = tmp_path / "segops.py"
    script.write_text(SEG_OPS_CHUNK_SCRIPT)
    env = dict(os.environ, GBSCAN_CHUNK_BYTES="4096", GBSCAN_CHUNK_LAG="2")
    r = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
