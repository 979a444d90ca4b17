"""Parity at the workload sizes the benchmark measures, every element checked
against the oracle.

- int32 n = 2^30, uniform [0, 255], inclusive and exclusive, and int64
  n = 2^29, uniform [0, 2^32): single-pass, two-pass and partitioned scans, each
  in the launch shape the benchmark takes for it (the tuned variant), bit-exact.
- fp32 n = 2^28, uniform [0, 1) on the 2^-24 grid and N(0, 1), plain and
  compensated: max_k |y_k - y_k^ref| / sum_{i<=k} |a_i| against the compensated
  FP64 oracle, within 1e-5 (plain) and 1e-6 (compensated).
- 65,536 segments with lengths log-uniform in [1, 2^16], exclusive, through the
  CUDA-graph path: int32 U[0, 3] bit-exact, fp32 U[0, 1) within 1e-5.
- [4096, 8192] fp32 N(0, 1): the row scan and its backward (suffix scan)
  within 1e-5.
- int32 n = 2^30 running maximum and minimum, every algorithm, bit-exact;
  int64 n = 2^29 running maximum and minimum and uint32 n = 2^30 sums, every
  algorithm, bit-exact; segmented maximum and minimum of the 65,536-segment
  batch, bit-exact.
- Stream compaction of int32 n = 2^30 with half the elements kept, bit-exact.

The measured errors are printed; with GBSCAN_PARITY_REPORT set to a path they
are also written there as JSON.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi, autotune
from paper_2312_14874_gb300.graphs import SegmentedScanGraph

pytestmark = pytest.mark.gpu

ALGOS = ("single_pass", "two_pass", "partitioned")
REPORT: dict = {}


def dev():
    return torch.device("cuda", 0)


def record(key, value):
    REPORT[key] = value
    print(f"[parity] {key}: {value}", flush=True)
    path = os.environ.get("GBSCAN_PARITY_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(REPORT, f, indent=1, sort_keys=True)


def tuned(fam, n, algo):
    return autotune.choose(fam, fam[5:], n, algo)[1]


@pytest.mark.parametrize("exclusive", [False, True])
def test_int32_2e30_every_algorithm(exclusive):
    n = 1 << 30
    a = synth.uniform_i32(n, 256, seed=0)
    want = oracle.scan_i32(a, exclusive)
    x = torch.from_numpy(a).to(dev())
    y = torch.empty_like(x)
    for algo in ALGOS:
        y.fill_(-1)
        gb.scan(x, exclusive, out=y, algo=algo, variant=tuned("scan_i32", n, algo))
        assert gb.device_status() == 0, algo
        assert np.array_equal(y.cpu().numpy(), want), algo
    record(f"i32_2^30_{'exclusive' if exclusive else 'inclusive'}", "bit-exact: " + ", ".join(ALGOS))


@pytest.mark.parametrize("op", ["max", "min"])
def test_int32_2e30_running_max_min(op):
    n = 1 << 30
    a = (synth.uniform_i32(n, 1 << 31, seed=0).astype(np.int64) - (1 << 30)).astype(np.int32)
    want = oracle.scan_op(a, op)
    x = torch.from_numpy(a).to(dev())
    y = torch.empty_like(x)
    for algo in ALGOS:
        y.fill_(0)
        gb.scan(x, out=y, op=op, algo=algo)
        assert gb.device_status() == 0, algo
        assert np.array_equal(y.cpu().numpy(), want), algo
    record(f"i32_2^30_running_{op}", "bit-exact: " + ", ".join(ALGOS))


def test_compact_int32_2e30_half_kept():
    """Every compaction variant (the partitioned one, which the tuned table
    takes at this size, and the single-pass one)."""
    n = 1 << 30
    a = synth.uniform_i32(n, 1 << 31, seed=1)
    f = (synth.unit_f32(n, seed=2) < 0.5).astype(np.uint8)
    want = oracle.compact(a, f)
    x, fl = torch.from_numpy(a).to(dev()), torch.from_numpy(f).to(dev())
    out = torch.empty_like(x)
    for v in range(gb.num_variants(torch.int32, _capi.KIND_COMPACT)):
        out.fill_(-1)
        _, cnt = gb.compact(x, fl, out=out, variant=v)
        k = int(cnt.item())
        assert k == want.size, v
        assert np.array_equal(out[:k].cpu().numpy(), want), v
    assert gb.device_status() == 0
    record("compact_i32_2^30_half_kept", f"bit-exact in every variant, kept {k}")


def test_int64_2e29_every_algorithm():
    n = 1 << 29
    a = synth.uniform_i64(n, 1 << 32, seed=0)
    want = oracle.scan_i64(a)
    x = torch.from_numpy(a).to(dev())
    y = torch.empty_like(x)
    for algo in ALGOS:
        y.fill_(-1)
        gb.scan(x, out=y, algo=algo, variant=tuned("scan_i64", n, algo))
        assert gb.device_status() == 0, algo
        assert np.array_equal(y.cpu().numpy(), want), algo
    record("i64_2^29_inclusive", "bit-exact: " + ", ".join(ALGOS))


def test_uint32_2e30_sums():
    """uint32 inclusive sums of 2^30 values spanning the whole range (the
    total wraps many times), tuned variant of every algorithm, bit-exact."""
    n = 1 << 30
    a = synth.uniform_i64(n, 1 << 32, seed=3).astype(np.uint32)
    want = oracle.scan_u32(a)
    x = torch.from_numpy(a.view(np.int32)).to(dev()).view(torch.uint32)
    y = torch.empty_like(x)
    for algo in ALGOS:
        y.view(torch.int32).fill_(-1)
        gb.scan(x, out=y, algo=algo, variant=tuned("scan_i32", n, algo))
        assert gb.device_status() == 0, algo
        assert np.array_equal(y.view(torch.int32).cpu().numpy().view(np.uint32), want), algo
    record("u32_2^30_inclusive", "bit-exact: " + ", ".join(ALGOS))


@pytest.mark.parametrize("op", ["max", "min"])
def test_int64_2e29_running_max_min(op):
    n = 1 << 29
    a = synth.uniform_i64(n, 1 << 32, seed=4).astype(np.int64) * 2_000_003 - (1 << 52)
    want = oracle.scan_op(a, op)
    x = torch.from_numpy(a).to(dev())
    y = torch.empty_like(x)
    for algo in ALGOS:
        y.fill_(0)
        gb.scan(x, out=y, op=op, algo=algo, variant=2)
        assert gb.device_status() == 0, algo
        assert np.array_equal(y.cpu().numpy(), want), algo
    record(f"i64_2^29_running_{op}", "bit-exact: " + ", ".join(ALGOS))


@pytest.mark.parametrize("op", ["max", "min"])
def test_segmented_65536_max_min(op):
    """Segmented running maximum / minimum of the 65,536-segment batch, int32,
    exclusive, bit-exact."""
    off = synth.segment_offsets(65536, max_log2=16, seed=0)
    n = int(off[-1])
    a = (synth.uniform_i32(n, 1 << 31, seed=5).astype(np.int64) - (1 << 30)).astype(np.int32)
    want = oracle.seg_scan_op(a, off, op, True)
    y = gb.segmented(torch.from_numpy(a).to(dev()), torch.from_numpy(off).to(dev()), True, op=op)
    assert gb.device_status() == 0
    assert np.array_equal(y.cpu().numpy(), want)
    record(f"seg_i32_65536_exclusive_{op}", f"bit-exact, n = {n}")


@pytest.mark.parametrize("dist", ["uniform", "normal"])
def test_fp32_2e28_errors(dist):
    n = 1 << 28
    a = synth.unit_f32(n, seed=0) if dist == "uniform" else synth.normal_f32(n, seed=0)
    ref = oracle.scan_f32_ref(a)
    den = oracle.abs_scan_f32(a)
    x = torch.from_numpy(a).to(dev())
    y = torch.empty_like(x)
    errs = {}
    for comp in (False, True):
        fam = "scan_f32c" if comp else "scan_f32"
        for algo in ALGOS:
            gb.inclusive(x, out=y, algo=algo, compensated=comp, variant=tuned(fam, n, algo))
            assert gb.device_status() == 0, (algo, comp)
            err, at = oracle.max_rel_err(y.cpu().numpy(), ref, den)
            errs[f"{'compensated' if comp else 'plain'}_{algo}"] = float(err)
            assert err <= (1e-6 if comp else 1e-5), (algo, comp, err, at)
    record(f"f32_2^28_{dist}_max_rel_err", errs)


@pytest.mark.parametrize("dtype", [torch.int32, torch.float32])
def test_segmented_65536_graph(dtype):
    off = synth.segment_offsets(65536, max_log2=16, seed=0)
    n = int(off[-1])
    if dtype == torch.int32:
        a = synth.uniform_i32(n, 4, seed=0)
    else:
        a = synth.unit_f32(n, seed=0)
    g = SegmentedScanGraph(n, off, dtype, exclusive=True, device=dev())
    y = g.run(torch.from_numpy(a).to(dev())).cpu().numpy()
    assert g.device_status() == 0
    if dtype == torch.int32:
        assert np.array_equal(y, oracle.seg_scan_i32(a, off, True))
        record("seg_i32_65536_exclusive", f"bit-exact, n={n}")
    else:
        err, at = oracle.max_rel_err(y, oracle.seg_scan_f32_ref(a, off, True),
                                     oracle.seg_abs_scan_f32(a, off, True))
        assert err <= 1e-5, (err, at)
        record("seg_f32_65536_exclusive_max_rel_err", float(err))


def test_rows_4096x8192_forward_and_backward():
    rows, cols = 4096, 8192
    a = synth.normal_f32(rows * cols, seed=0).reshape(rows, cols)
    x = torch.from_numpy(a).to(dev())
    y = gb.rows(x).cpu().numpy()
    den = oracle.rows_scan_f32_ref(np.abs(a))
    err_f, at = oracle.max_rel_err(y, oracle.rows_scan_f32_ref(a), den)
    assert err_f <= 1e-5, (err_f, at)
    g = synth.normal_f32(rows * cols, seed=1).reshape(rows, cols)
    dx = gb.backward(torch.from_numpy(g).to(dev())).cpu().numpy()
    err_b, at = oracle.max_rel_err(dx, oracle.rows_suffix_f32_ref(g), oracle.rows_suffix_abs_f32(g))
    assert err_b <= 1e-5, (err_b, at)
    assert gb.device_status() == 0
    record("rows_f32_4096x8192_max_rel_err", {"forward": float(err_f), "backward": float(err_b)})
