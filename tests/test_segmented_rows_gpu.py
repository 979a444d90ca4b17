"""GPU parity for the batched segmented scan, the row-wise scan along the last
dim, and its gradient (reverse suffix scan), against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def random_offsets(n_seg, seed, max_len, empty_frac=0.1):
    lens = synth.uniform_i64(n_seg, max_len + 1, seed=seed, stream=1)
    drop = synth.unit_f32(n_seg, seed=seed, stream=2) < empty_frac
    lens = np.where(drop, 0, lens)
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)


OFFSET_CASES = {
    "tiny_with_empties": lambda: random_offsets(3000, 1, 40, 0.3),
    "mixed": lambda: random_offsets(500, 2, 20000, 0.1),
    "log_uniform_small": lambda: synth.segment_offsets(4000, max_log2=12, seed=3),
    "one_segment": lambda: np.array([0, 3 * 5120 + 17], dtype=np.int64),
    "all_length_one": lambda: np.arange(20000 + 1, dtype=np.int64),
    "long_segments": lambda: np.array([0, 1, 70000, 70001, 200000, 200000, 250003], np.int64),
    "trailing_empty": lambda: np.array([0, 10, 5000, 12000, 12000, 12000], np.int64),
    "leading_empty": lambda: np.array([0, 0, 0, 9000, 9001], np.int64),
}


@pytest.mark.parametrize("case", sorted(OFFSET_CASES))
@pytest.mark.parametrize("dtype_key", ["i32", "f32"])
def test_segmented(case, dtype_key):
    off = OFFSET_CASES[case]()
    n = int(off[-1])
    torch_dt = torch.int32 if dtype_key == "i32" else torch.float32
    a = synth.uniform_i32(n, 4, seed=5) if dtype_key == "i32" else synth.unit_f32(n, seed=5)
    x, o = to_dev(a), to_dev(off)
    for v in range(gb.num_variants(torch_dt, _capi.KIND_SEGMENTED)):
        for excl in (False, True):
            y = gb.segmented(x, o, exclusive=excl, variant=v).cpu().numpy()
            if dtype_key == "i32":
                assert np.array_equal(y, oracle.seg_scan_i32(a, off, excl)), (v, excl)
            else:
                err, k = oracle.max_rel_err(y, oracle.seg_scan_f32_ref(a, off, excl),
                                            oracle.seg_abs_scan_f32(a, off, excl))
                assert err <= 1e-5, (v, excl, err, k)
    assert gb.device_status() == 0


SEG_PARTITION_SCRIPT = r"""
import sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi
dev = torch.device("cuda", 0)
def random_offsets(n_seg, seed, max_len, empty_frac):
    lens = synth.uniform_i64(n_seg, max_len + 1, seed=seed, stream=1)
    drop = synth.unit_f32(n_seg, seed=seed, stream=2) < empty_frac
    lens = np.where(drop, 0, lens)
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
cases = {
    "mixed": random_offsets(400, 12, 20000, 0.1),
    "spanning_chunks": np.array([0, 1, 700000, 700001, 2000000, 2000000, 2100007], np.int64),
    "length_one": np.arange(200000 + 1, dtype=np.int64),
    "log_uniform": synth.segment_offsets(3000, max_log2=12, seed=13),
}
for name, off in cases.items():
    n = int(off[-1])
    o = torch.from_numpy(off).to(dev)
    for key in ("i32", "f32"):
        dt = torch.int32 if key == "i32" else torch.float32
        a = synth.uniform_i32(n, 4, seed=7) if key == "i32" else synth.unit_f32(n, seed=7)
        x = torch.from_numpy(a).to(dev)
        for v in range(gb.num_variants(dt, _capi.KIND_SEGMENTED)):
            if gb.variant_info(dt, _capi.KIND_SEGMENTED, v)["threads"] != \
                    (gb.variant_info(dt, _capi.KIND_SEGMENTED, v)["tile"] //
                     gb.variant_info(dt, _capi.KIND_SEGMENTED, v)["items"] + 64):
                continue  # the single-pass variants: no chunks
            for excl in (False, True):
                y = gb.segmented(x, o, exclusive=excl, variant=v).cpu().numpy()
                if key == "i32":
                    assert np.array_equal(y, oracle.seg_scan_i32(a, off, excl)), (name, v, excl)
                else:
                    err, k = oracle.max_rel_err(y, oracle.seg_scan_f32_ref(a, off, excl),
                                                oracle.seg_abs_scan_f32(a, off, excl))
                    assert err <= 1e-5, (name, v, excl, err, k)
assert gb.device_status() == 0
print("ok")
"""


@pytest.mark.parametrize("lag", [1, 3])
def test_segmented_partitioned_small_chunks(tmp_path, lag):
    """The segmented scan's partitioned variants with 16-tile chunks (set in a
    child process): segments spanning many chunks, a head on every element,
    empty segments; the head flags travel through the tile sums, the chunk
    scan's offsets and the chained chunk prefixes."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    script = tmp_path / "segpart.py"
    script.write_text(SEG_PARTITION_SCRIPT)
    env = dict(os.environ, GBSCAN_CHUNK_BYTES="4096", GBSCAN_CHUNK_LAG=str(lag))
    r = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


def test_segmented_bad_offsets_reported():
    n = 10000
    x = torch.zeros(n, dtype=torch.int32, device=dev())
    for bad in ([0, 6000, 5000, n], [1, 5000, n], [0, 5000, n - 1]):
        gb.segmented(x, to_dev(np.array(bad, np.int64)))
        assert gb.device_status() == _capi.ERR_INVALID_ARG
    gb.segmented(x, to_dev(np.array([0, 5000, n], np.int64)))
    assert gb.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(1, 1), (3, 1), (1, 5121), (7, 33), (64, 1000), (5, 20000),
                                   (1000, 3), (40, 8192), (37, 1000), (3, 8960), (2, 10753),
                                   (9, 4480), (2, 4481), (4096, 1024), (513, 4096)])
def test_rows_and_backward(dtype, shape):
    """Every variant, inclusive and exclusive, forward and backward.  Rows that
    fit a variant's row-block tile (fp32 8960 / 10752 / 10240 elements, fp64
    4480 / 5376 / 5120) take the row-block kernel, several rows to an item when
    they are short, with a partial last item; longer rows (20000, 10753 fp32,
    4481+ fp64) take the chained kernel with row heads.  Row lengths that are
    not 16-byte multiples take the element-wise load path."""
    rows, cols = shape
    g = (synth.normal_f32 if dtype == torch.float32 else synth.normal_f64)(rows * cols, seed=9)
    g = g.reshape(rows, cols)
    x = to_dev(g)
    tol = 1e-5 if dtype == torch.float32 else 1e-13
    for v in range(gb.num_variants(dtype, _capi.KIND_ROWS)):
        for excl in (False, True):
            # forward: per-row scan = segmented scan with uniform segments
            y = gb.rows(x, exclusive=excl, variant=v).cpu().numpy()
            if dtype == torch.float32:
                off = np.arange(rows + 1, dtype=np.int64) * cols
                ref = oracle.seg_scan_f32_ref(g.reshape(-1), off, excl).reshape(rows, cols)
                den = oracle.seg_abs_scan_f32(g.reshape(-1), off, excl).reshape(rows, cols)
            else:
                ref = np.stack([oracle.scan_f64_ref(r, excl) for r in g])
                den = np.stack([oracle.scan_f64_ref(np.abs(r), excl) for r in g])
            err, k = oracle.max_rel_err(y, ref, den)
            assert err <= tol, ("fwd", v, excl, err, k)
            # backward: reverse suffix scan
            d = gb.backward(x, exclusive=excl, variant=v).cpu().numpy()
            if dtype == torch.float32:
                ref = oracle.rows_suffix_f32_ref(g, excl)
                den = oracle.rows_suffix_abs_f32(g, excl)
            else:
                ref = oracle.rows_suffix_f64_ref(g, excl)
                den = oracle.rows_suffix_f64_ref(np.abs(g), excl)
            err, k = oracle.max_rel_err(d, ref, den)
            assert err <= tol, ("bwd", v, excl, err, k)


def test_backward_ones_closed_form():
    rows, cols = 16, 9000
    g = torch.ones(rows, cols, device=dev())
    d = gb.backward(g)
    want = (cols - torch.arange(cols, device=dev(), dtype=torch.float32)).expand(rows, cols)
    assert torch.equal(d, want)
    d = gb.backward(g, exclusive=True)
    assert torch.equal(d, want - 1)


def test_backward_in_place():
    rows, cols = 33, 7001
    g = synth.normal_f32(rows * cols, seed=4).reshape(rows, cols)
    x = to_dev(g)
    gb.backward(x, out=x)
    err, _ = oracle.max_rel_err(x.cpu().numpy(), oracle.rows_suffix_f32_ref(g),
                                oracle.rows_suffix_abs_f32(g))
    assert err <= 1e-5
