"""GPU parity: the CUDA scans against the CPU oracle, element by element.

Integers must match bit for bit.  Floats are compared with the error metric
max_k |y_k - y_k^FP64| / sum_{i<=k} |a_i| against the FP64 oracle:
<= 1e-5 for plain fp32, <= 1e-6 for compensated fp32, <= 1e-13 for fp64.
Sizes span several tiles of every variant plus ragged tails; edge cases cover
n = 0 and 1, tile boundaries, in-place, and misaligned pointers.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
TOL_F32C = 1e-6
TOL_F64 = 1e-13

SIZES = [1, 2, 31, 32, 33, 1535, 1536, 1537, 3071, 3072, 3073, 5119, 5120, 5121, 10239, 10240,
         10241, 3 * 5120 + 77, 100_003, (1 << 20) + 7]


def dev():
    return torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def variants(dtype, kind=_capi.KIND_SCAN):
    return list(range(gb.num_variants(dtype, kind)))


def gen(dtype_key, n, seed):
    if dtype_key == "i32":
        return synth.uniform_i32(n, 256, seed=seed)
    if dtype_key == "i64":
        return synth.uniform_i64(n, 1 << 32, seed=seed)
    if dtype_key == "f32":
        return synth.normal_f32(n, seed=seed)
    return synth.normal_f64(n, seed=seed)


def check(dtype_key, a, y, excl, compensated=False):
    if dtype_key == "i32":
        assert np.array_equal(y, oracle.scan_i32(a, excl))
    elif dtype_key == "i64":
        assert np.array_equal(y, oracle.scan_i64(a, excl))
    elif dtype_key == "f32":
        ref = oracle.scan_f32_ref(a, excl)
        den = oracle.abs_scan_f32(a, excl)
        err, k = oracle.max_rel_err(y, ref, den)
        assert err <= (TOL_F32C if compensated else TOL_F32), (err, k)
    else:
        ref = oracle.scan_f64_ref(a, excl)
        den = oracle.scan_f64_ref(np.abs(a), excl)
        err, k = oracle.max_rel_err(y, ref, den)
        assert err <= TOL_F64, (err, k)


@pytest.mark.parametrize("dtype_key", ["i32", "i64", "f32", "f64"])
@pytest.mark.parametrize("algo", ["single_pass", "two_pass", "partitioned"])
def test_scan_sizes_all_variants(dtype_key, algo):
    torch_dt = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32,
                "f64": torch.float64}[dtype_key]
    for v in variants(torch_dt):
        for n in SIZES:
            a = gen(dtype_key, n, seed=n)
            x = to_dev(a)
            for excl in (False, True):
                y = gb.scan(x, excl, algo=algo, variant=v).cpu().numpy()
                check(dtype_key, a, y, excl)
    assert gb.device_status() == 0


# The resident scan: one block per tile (5120 4-byte or 2560 8-byte elements),
# every block resident at once, so at most SMs x blocks-per-SM tiles.
def resident_limit(dtype_key, compensated=False):
    torch_dt = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32,
                "f64": torch.float64}[dtype_key]
    lim = gb.resident_max_n(torch_dt, compensated=compensated)
    sms = torch.cuda.get_device_properties(dev()).multi_processor_count
    tile = 2560 if dtype_key in ("i64", "f64") else 5120
    assert lim % (sms * tile) == 0 and 1 <= lim // (sms * tile) <= 8
    return lim


@pytest.mark.parametrize("dtype_key", ["i32", "i64", "f32", "f64"])
def test_scan_resident(dtype_key):
    """The size ladder, the largest input the resident scan takes, and one
    element more (refused with UNSUPPORTED, nothing launched); inclusive and
    exclusive, in place, plain and compensated, and a misaligned view (the
    lanes' copies and stores on every tile)."""
    for comp in ((False, True) if dtype_key == "f32" else (False,)):
        lim = resident_limit(dtype_key, comp)
        for n in SIZES + [lim - 1, lim]:
            a = gen(dtype_key, n, seed=n)
            x = to_dev(a)
            for excl in (False, True):
                y = gb.scan(x, excl, algo="resident", variant=0, compensated=comp).cpu().numpy()
                check(dtype_key, a, y, excl, compensated=comp)
            x2 = x.clone()
            gb.scan(x2, out=x2, algo="resident", variant=0, compensated=comp)
            check(dtype_key, a, x2.cpu().numpy(), False, compensated=comp)
        x = torch.zeros(lim + 1, dtype=x.dtype, device=dev())
        with pytest.raises(_capi.GbscanError) as e:
            gb.scan(x, algo="resident", variant=0, compensated=comp)
        assert e.value.status == _capi.ERR_UNSUPPORTED
    a = gen(dtype_key, 3 * 5120 + 9, seed=5)
    xb = to_dev(a)[1:]
    y = gb.scan(xb, algo="resident", variant=0).cpu().numpy()
    check(dtype_key, a[1:], y, False)
    assert gb.device_status() == 0


@pytest.mark.parametrize("algo", ["single_pass", "two_pass", "partitioned"])
def test_scan_f32_compensated(algo):
    for v in variants(torch.float32):
        for n in SIZES:
            for dist in ("normal", "unit"):
                a = synth.normal_f32(n, seed=n) if dist == "normal" else synth.unit_f32(n, seed=n)
                x = to_dev(a)
                for excl in (False, True):
                    y = gb.scan(x, excl, algo=algo, variant=v, compensated=True).cpu().numpy()
                    check("f32", a, y, excl, compensated=True)


def test_closed_forms_on_gpu():
    n = (1 << 22) + 3
    ones = torch.ones(n, dtype=torch.int32, device=dev())
    k = torch.arange(n, dtype=torch.int64, device=dev())
    assert torch.equal(gb.inclusive(ones).long(), k + 1)
    assert torch.equal(gb.exclusive(ones).long(), k)
    tri = gb.inclusive(k)
    assert torch.equal(tri, k * (k + 1) // 2)
    # int32 wraps: low 32 bits of the int64 result
    t32 = gb.inclusive(k.to(torch.int32)).cpu().numpy()
    want = ((k.cpu().numpy() * (k.cpu().numpy() + 1) // 2) % (1 << 32)).astype(np.uint32)
    assert np.array_equal(t32.view(np.uint32), want)


@pytest.mark.parametrize("dtype_key", ["i32", "i64", "f32"])
def test_in_place(dtype_key):
    n = 5 * 5120 + 13
    a = gen(dtype_key, n, seed=7)
    for algo in ("single_pass", "two_pass", "partitioned"):
        for excl in (False, True):
            x = to_dev(a)
            y = gb.scan(x, excl, out=x, algo=algo)
            assert y.data_ptr() == x.data_ptr()
            check(dtype_key, a, x.cpu().numpy(), excl)


@pytest.mark.parametrize("dtype_key", ["i32", "i64", "f32"])
def test_misaligned_pointers(dtype_key):
    """Slices at element offsets 1..3 are not 16-byte aligned: the element-wise
    load/store path must give the same results."""
    n = 4 * 5120 + 5
    torch_dt = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32}[dtype_key]
    for off_in, off_out in ((1, 0), (0, 3), (2, 1), (3, 3)):
        a = gen(dtype_key, n, seed=off_in * 4 + off_out)
        big_in = torch.zeros(n + 8, dtype=torch_dt, device=dev())
        big_out = torch.zeros(n + 8, dtype=torch_dt, device=dev())
        big_in[off_in:off_in + n] = to_dev(a)
        x = big_in[off_in:off_in + n]
        y = big_out[off_out:off_out + n]
        for excl in (False, True):
            gb.scan(x, excl, out=y)
            check(dtype_key, a, y.cpu().numpy(), excl)
        # guard zones untouched
        assert torch.count_nonzero(big_out[:off_out]) == 0
        assert torch.count_nonzero(big_out[off_out + n:]) == 0


def test_canary_guard_zones():
    """The kernels write exactly [out, out + n): 4 KiB canaries on both sides
    and around the workspace survive."""
    n = 7 * 5120 + 99
    pad = 1024
    a = synth.uniform_i32(n, 16, seed=3)
    buf = torch.full((n + 2 * pad,), -123456, dtype=torch.int32, device=dev())
    x = to_dev(a)
    out = buf[pad:pad + n]
    ws_need = gb.workspace_bytes(torch.int32, _capi.KIND_SCAN, n)
    wsbuf = torch.zeros(ws_need + 2 * 4096, dtype=torch.uint8, device=dev())
    wsbuf[:4096] = 0xAB
    wsbuf[4096 + ws_need:] = 0xCD
    L = _capi.lib()
    s = torch.cuda.current_stream().cuda_stream
    wptr = wsbuf.data_ptr() + 4096
    for algo in (1, 2, 3):
        assert L.scan_inclusive_i32(x.data_ptr(), out.data_ptr(), n, wptr, ws_need, algo, 0, s) == 0
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.scan_i32(a))
    assert torch.all(buf[:pad] == -123456) and torch.all(buf[pad + n:] == -123456)
    assert torch.all(wsbuf[:4096] == 0xAB) and torch.all(wsbuf[4096 + ws_need:] == 0xCD)
    assert L.scan_get_device_status(wptr, s) == 0


def test_raw_c_abi_statuses_on_gpu():
    L = _capi.lib()
    s = torch.cuda.current_stream().cuda_stream
    x = torch.zeros(1000, dtype=torch.int32, device=dev())
    ws = gb.Workspace(4096)
    assert L.scan_inclusive_i32(x.data_ptr(), x.data_ptr(), 1000, ws.ptr, ws.nbytes, 0, 0, s) == 0
    assert L.scan_inclusive_i32(x.data_ptr(), x.data_ptr() + 4, 999, ws.ptr, ws.nbytes, 0, 0,
                                s) == _capi.ERR_INVALID_ARG
    assert L.scan_inclusive_i32(x.data_ptr(), x.data_ptr(), 1000, ws.ptr, 300, 0, 0, s) == \
        _capi.ERR_WORKSPACE
    assert L.scan_get_device_status(ws.ptr, s) == 0


def test_many_launches_reuse_workspace():
    """The epoch tags make stale status words invalid: alternating sizes and
    dtypes on one workspace never mixes up tiles."""
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_SCAN, 1 << 21))
    rng_sizes = [1 << 21, 5000, 1 << 20, 123457, 1 << 21, 77, 400_000]
    for i, n in enumerate(rng_sizes * 3):
        a = synth.uniform_i32(n, 1 << 20, seed=100 + i)
        y = gb.inclusive(to_dev(a), workspace=ws).cpu().numpy()
        assert np.array_equal(y, oracle.scan_i32(a))
        b = synth.uniform_i64(n // 2 + 1, 1 << 32, seed=200 + i)
        z = gb.exclusive(to_dev(b), workspace=ws).cpu().numpy()
        assert np.array_equal(z, oracle.scan_i64(b, True))
    assert gb.device_status(ws) == 0


PARTITION_SCRIPT = r"""
import sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_2312_14874_gb300 as gb
dev = torch.device("cuda", 0)
# 16-tile chunks (the smallest): many chunk boundaries and a ragged last chunk
for key, n in (("i32", 16 * 5120 * 37 + 99), ("i64", 16 * 2560 * 21 + 5), ("f32", 16 * 5120 * 9 + 7),
               ("f64", 16 * 2560 * 5 + 3)):
    for v in range(gb.num_variants({"i32": torch.int32, "i64": torch.int64, "f32": torch.float32,
                                    "f64": torch.float64}[key])):
        if key == "i32":
            a = synth.uniform_i32(n, 1 << 20, seed=v)
        elif key == "i64":
            a = synth.uniform_i64(n, 1 << 32, seed=v)
        elif key == "f32":
            a = synth.normal_f32(n, seed=v)
        else:
            a = synth.normal_f64(n, seed=v)
        x = torch.from_numpy(a).to(dev)
        for excl in (False, True):
            y = gb.scan(x, excl, algo="partitioned", variant=v).cpu().numpy()
            if key == "i32":
                assert np.array_equal(y, oracle.scan_i32(a, excl)), (key, v, excl)
            elif key == "i64":
                assert np.array_equal(y, oracle.scan_i64(a, excl)), (key, v, excl)
            elif key == "f32":
                err, _ = oracle.max_rel_err(y, oracle.scan_f32_ref(a, excl), oracle.abs_scan_f32(a, excl))
                assert err <= 1e-5, (key, v, excl, err)
            else:
                err, _ = oracle.max_rel_err(y, oracle.scan_f64_ref(a, excl),
                                            oracle.scan_f64_ref(np.abs(a), excl))
                assert err <= 1e-13, (key, v, excl, err)
assert gb.device_status() == 0
print("ok")
"""


@pytest.mark.parametrize("lag", [1, 2, 5])
def test_partitioned_many_small_chunks(tmp_path, lag):
    """The partitioned scan with the smallest chunks (16 tiles, set through
    GBSCAN_CHUNK_BYTES in a child process): dozens of chunk prefixes chained,
    with the second pass of a chunk 1, 2 or 5 chunks behind its first pass
    (GBSCAN_CHUNK_LAG)."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    script = tmp_path / "part.py"
    script.write_text(PARTITION_SCRIPT)
    env = dict(os.environ, GBSCAN_CHUNK_BYTES="4096", GBSCAN_CHUNK_LAG=str(lag))
    r = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def test_partitioned_multi_chunk_default_size():
    """Default chunks (8 MiB): an array of several chunks plus a ragged tail."""
    n = 7 * 1228 * 5120 + 12345
    a = synth.uniform_i32(n, 256, seed=11)
    x = to_dev(a)
    for excl in (False, True):
        y = gb.scan(x, excl, algo="partitioned").cpu().numpy()
        assert np.array_equal(y, oracle.scan_i32(a, excl))
