"""Ordering stress, bounded waits, CUDA-graph replay and autograd on the GPU.

No test here faults or hangs the GPU: the "dropped tile" case makes one tile
skip its status publication, and its successor's bounded wait (a 2 ms limit
set in the workspace header) runs out and records GBSCAN_ERR_TIMEOUT, which
the host reads back; the kernel finishes normally.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi
from paper_2312_14874_gb300.graphs import SegmentedScanGraph

pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def test_race_stress_random_publication_delays():
    """Pseudo-random sleeps before every status publication reorder tile
    completion; integer results must stay bit-exact over many repetitions,
    with far more tiles than resident blocks."""
    n = 600 * 5120 + 333
    a = synth.uniform_i32(n, 1 << 16, seed=1)
    want = oracle.scan_i32(a)
    x = to_dev(a)
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_SCAN, n))
    gb.set_debug(delay_ns_max=3000, workspace=ws)
    for rep in range(40):
        v = rep % gb.num_variants(torch.int32)
        y = gb.inclusive(x, variant=v, workspace=ws, algo="single_pass").cpu().numpy()
        assert gb.device_status(ws) == 0, (rep, v)
        assert np.array_equal(y, want), (rep, v)
    gb.set_debug(workspace=ws)
    assert gb.device_status(ws) == 0


def test_race_stress_segmented_and_i64():
    off = synth.segment_offsets(3000, max_log2=12, seed=2)
    n = int(off[-1])
    a = synth.uniform_i32(n, 4, seed=3)
    # one workspace for both kinds: the larger of the two sizes
    ws = gb.Workspace(max(gb.workspace_bytes(torch.int64, _capi.KIND_SCAN, n),
                          gb.workspace_bytes(torch.int32, _capi.KIND_SEGMENTED, n, off.size - 1)))
    gb.set_debug(delay_ns_max=2000, workspace=ws)
    x, o = to_dev(a), to_dev(off)
    want = oracle.seg_scan_i32(a, off, True)
    b = synth.uniform_i64(n, 1 << 32, seed=4)
    want64 = oracle.scan_i64(b)
    xb = to_dev(b)
    for rep in range(15):
        v = rep % gb.num_variants(torch.int32, _capi.KIND_SEGMENTED)
        assert np.array_equal(gb.segmented(x, o, exclusive=True, workspace=ws, variant=v)
                              .cpu().numpy(), want), rep
        assert gb.device_status(ws) == 0, rep
        assert np.array_equal(gb.inclusive(xb, workspace=ws, variant=rep % 5, algo="single_pass")
                              .cpu().numpy(), want64), rep
        assert gb.device_status(ws) == 0, rep
    gb.set_debug(workspace=ws)
    assert gb.device_status(ws) == 0


PARTITION_STRESS = r"""
import sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi
dev = torch.device("cuda", 0)
n = 16 * 5120 * 23 + 777
a = synth.uniform_i32(n, 1 << 16, seed=9)
want_in, want_ex = oracle.scan_i32(a, False), oracle.scan_i32(a, True)
b = synth.uniform_i64(n // 2, 1 << 32, seed=10)
want64 = oracle.scan_i64(b)
x, xb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
ws = gb.Workspace(gb.workspace_bytes(torch.int64, _capi.KIND_SCAN, n))
gb.set_debug(delay_ns_max=3000, workspace=ws)
for rep in range(24):
    v = rep % gb.num_variants(torch.int32)
    excl = rep % 2 == 1
    y = gb.scan(x, excl, workspace=ws, algo="partitioned", variant=v).cpu().numpy()
    assert gb.device_status(ws) == 0, (rep, v)
    assert np.array_equal(y, want_ex if excl else want_in), (rep, v)
    y = gb.inclusive(xb, workspace=ws, algo="partitioned", variant=v).cpu().numpy()
    assert gb.device_status(ws) == 0, (rep, v)
    assert np.array_equal(y, want64), (rep, v)
gb.set_debug(workspace=ws)
assert gb.device_status(ws) == 0
print("ok")
"""


@pytest.mark.parametrize("lag", [1, 3])
def test_race_stress_partitioned_small_chunks(tmp_path, lag):
    """Pseudo-random sleeps before every tile-sum and chunk-prefix publication
    of the partitioned scan, with 16-tile chunks (set in a child process):
    dozens of chunk scans and chained chunk prefixes reordered in time, results
    bit-exact on every repetition."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    script = tmp_path / "stress.py"
    script.write_text(PARTITION_STRESS)
    env = dict(os.environ, GBSCAN_CHUNK_BYTES="4096", GBSCAN_CHUNK_LAG=str(lag))
    r = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


EPOCH_MASK = (1 << 29) - 1  # status words carry a 29-bit launch epoch


def test_epoch_wrap_every_algorithm():
    """Launches across the epoch wrap (the workspace header's epoch set just
    below 2^29 - 1): the wrapping launch clears every status word and the
    launches after it start from epoch 1.  Every algorithm (the resident scan,
    whose last block makes its epoch the completed one, included), int32 and
    int64, and the segmented scan stay exact, with no device error."""
    n = 40 * 7168 + 999
    a = synth.uniform_i32(n, 1 << 16, seed=31)
    b = synth.uniform_i64(n, 1 << 32, seed=32)
    off = synth.segment_offsets(200, max_log2=12, seed=33)
    sg = synth.uniform_i32(int(off[-1]), 4, seed=34)
    x, xb = torch.from_numpy(a).to(dev()), torch.from_numpy(b).to(dev())
    xs, o = torch.from_numpy(sg).to(dev()), torch.from_numpy(off).to(dev())
    want, want64 = oracle.scan_i32(a), oracle.scan_i64(b)
    wants = oracle.seg_scan_i32(sg, off, True)
    ws = gb.Workspace(gb.workspace_bytes(torch.int64, _capi.KIND_SEGMENTED, n, off.size - 1))
    for algo in ("resident", "single_pass", "two_pass", "partitioned"):
        ws.buf[0:4].view(torch.int32).fill_(EPOCH_MASK - 2)  # the last completed epoch
        for rep in range(5):  # epochs 2^29 - 2, 2^29 - 1 (the wrap), 1, 2, 3
            y = gb.inclusive(x, workspace=ws, algo=algo).cpu().numpy()
            assert np.array_equal(y, want), (algo, rep)
            y = gb.inclusive(xb, workspace=ws, algo=algo).cpu().numpy()
            assert np.array_equal(y, want64), (algo, rep)
            y = gb.segmented(xs, o, exclusive=True, workspace=ws).cpu().numpy()
            assert np.array_equal(y, wants), (algo, rep)
        assert int(ws.buf[0:4].view(torch.int32).item()) < 64, algo  # wrapped
        assert gb.device_status(ws) == 0, algo


def test_epoch_wrap_compaction():
    """Stream compaction across the epoch wrap, every variant (the partitioned
    and the single-pass compaction): exact outputs and counts, the wrapping
    launch clears the status words, no device error."""
    n = 40 * 5120 + 999
    a = synth.uniform_i32(n, 1 << 30, seed=35)
    f = (synth.unit_f32(n, seed=36) < 0.4).astype(np.uint8)
    want = oracle.compact(a, f)
    x, fl = torch.from_numpy(a).to(dev()), torch.from_numpy(f).to(dev())
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_COMPACT, n))
    for v in range(gb.num_variants(torch.int32, _capi.KIND_COMPACT)):
        ws.buf[0:4].view(torch.int32).fill_(EPOCH_MASK - 2)  # the last completed epoch
        for rep in range(5):  # epochs 2^29 - 2, 2^29 - 1 (the wrap), 1, 2, 3
            out, cnt = gb.compact(x, fl, workspace=ws, variant=v)
            k = int(cnt.item())
            assert k == want.size and np.array_equal(out[:k].cpu().numpy(), want), (v, rep)
        assert int(ws.buf[0:4].view(torch.int32).item()) < 64, v  # wrapped
        assert gb.device_status(ws) == 0, v


PREFETCH_CHECK = r"""
import sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import oracle, synth
import paper_2312_14874_gb300 as gb
from paper_2312_14874_gb300 import _capi
dev = torch.device("cuda", 0)
n = 600 * 7168 + 1234   # several waves of tiles and a ragged tail
a = synth.uniform_i32(n, 1 << 16, seed=21)
x = torch.from_numpy(a).to(dev)
ws = gb.Workspace(gb.workspace_bytes(torch.int64, _capi.KIND_SCAN, n))
want = oracle.scan_i32(a)
for algo in ("single_pass", "partitioned"):
    for v in range(gb.num_variants(torch.int32)):
        y = gb.inclusive(x, workspace=ws, algo=algo, variant=v).cpu().numpy()
        assert np.array_equal(y, want), (algo, v)
b = synth.uniform_i64(n, 1 << 32, seed=22)
y = gb.inclusive(torch.from_numpy(b).to(dev), workspace=ws, algo="single_pass").cpu().numpy()
assert np.array_equal(y, oracle.scan_i64(b))
f = (synth.uniform_i32(n, 2, seed=23)).astype(np.uint8)
for v in range(gb.num_variants(torch.int32, _capi.KIND_COMPACT)):
    out, cnt = gb.compact(x, torch.from_numpy(f).to(dev), workspace=ws, variant=v)
    k = int(cnt.item())
    assert np.array_equal(out[:k].cpu().numpy(), oracle.compact(a, f)), v
off = synth.segment_offsets(300, max_log2=14, seed=24)
s_ = synth.uniform_i32(int(off[-1]), 4, seed=25)
for v in range(gb.num_variants(torch.int32, _capi.KIND_SEGMENTED)):
    ys = gb.segmented(torch.from_numpy(s_).to(dev), torch.from_numpy(off).to(dev), exclusive=True,
                      variant=v).cpu().numpy()
    assert np.array_equal(ys, oracle.seg_scan_i32(s_, off, True)), v
assert gb.device_status(ws) == 0
print("ok")
"""


@pytest.mark.parametrize("pf_bytes", ["1", "65536", "1073741824"])
def test_prefetch_distance_changes_no_result(tmp_path, pf_bytes):
    """The L2 prefetch ahead of the claims is a hint: with it off (1), at one
    tile ahead or less (64 KiB), and past the end of every input (1 GiB), the
    single-pass, partitioned, compaction and segmented kernels give the
    oracle's results (set in a child process: the distance is read once)."""
    import os
    import subprocess
    import sys
    from conftest import ROOT
    script = tmp_path / "prefetch.py"
    script.write_text(PREFETCH_CHECK)
    env = dict(os.environ, GBSCAN_PREFETCH_BYTES=pf_bytes)
    r = subprocess.run([sys.executable, str(script), ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr


# With a 2 ms spin limit, a launch that runs into a bounded wait must end
# within its normal time plus the bounds it can meet in sequence: the first
# wait to run out (a look-back or status wait: one spin limit; a pipeline wait:
# 4 spin limits + 10 ms) aborts the launch, the claim counter is poisoned, and
# every other wait then gives up within about 160 us.  One second is far above
# that and far below what a wait that ignored the abort would cost.
LAUNCH_BOUND_S = 1.0


@pytest.mark.parametrize("algo", ["single_pass", "partitioned", "two_pass", "resident"])
@pytest.mark.parametrize("dtype", [torch.int32, torch.int64, torch.float32])
def test_dropped_tile_times_out_and_recovers(dtype, algo):
    """A tile that never publishes (the drop hook) makes the waits on it run out:
    the single-pass look-back of later tiles, or the partitioned scan's chunk
    scan and the second pass behind it; in the two-pass scan, whose blocks
    never wait for one another, the hook instead leaves the tile's stage load
    unissued, so that stage never fills.  The launch ends with TIMEOUT recorded,
    within the bound above, and the same workspace works again once the hook is
    removed."""
    import time
    n = 50 * 5120
    ws = gb.Workspace(gb.workspace_bytes(dtype, _capi.KIND_SCAN, n))
    x = torch.ones(n, dtype=dtype, device=dev())
    gb.set_debug(spin_limit_us=2000, drop_tile=17, workspace=ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gb.inclusive(x, workspace=ws, algo=algo)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < LAUNCH_BOUND_S
    assert gb.device_status(ws) == _capi.ERR_TIMEOUT
    assert gb.device_status(ws) == 0  # cleared by the read
    # the workspace is usable again once the hook is removed
    gb.set_debug(workspace=ws)
    y = gb.inclusive(x, workspace=ws, algo=algo)
    assert torch.equal(y.long(), torch.arange(1, n + 1, device=dev()))
    assert gb.device_status(ws) == 0


def test_compact_dropped_tile_times_out_and_recovers():
    """Stream compaction, every variant (the partitioned one and the one on the
    single-pass look-back): a tile whose kept count is never published makes
    the waits on it run out; the launch ends within the bound with TIMEOUT and
    writes nothing outside the output, and the workspace works again once the
    hook is removed."""
    import time
    n = 50 * 5120
    x = torch.arange(n, dtype=torch.int32, device=dev())
    f = torch.ones(n, dtype=torch.uint8, device=dev())
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_COMPACT, n))
    for v in range(gb.num_variants(torch.int32, _capi.KIND_COMPACT)):
        ob = torch.full((n + 2,), -7, dtype=torch.int32, device=dev())
        gb.set_debug(spin_limit_us=2000, drop_tile=17, workspace=ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gb.compact(x, f, out=ob[1:n + 1], workspace=ws, variant=v)
        torch.cuda.synchronize()
        assert time.perf_counter() - t0 < LAUNCH_BOUND_S, v
        assert gb.device_status(ws) == _capi.ERR_TIMEOUT, v
        assert int(ob[0].item()) == -7 and int(ob[n + 1].item()) == -7, v
        gb.set_debug(workspace=ws)
        out, cnt = gb.compact(x, f, workspace=ws, variant=v)
        assert int(cnt.item()) == n and torch.equal(out, x), v
        assert gb.device_status(ws) == 0, v


def test_two_pass_compensated_stage_never_fills():
    """The compensated fp32 two-pass scan (AUTO's pick at 2^22) with one stage
    load never issued, at 2^22 elements (hundreds of tiles per block): the block whose
    stage never fills stops at once instead of paying the bound on every later
    tile; both passes end within the bound with TIMEOUT, and the next call on
    the same workspace is correct again."""
    import time
    n = 1 << 22
    ws = gb.Workspace(gb.workspace_bytes(torch.float32, _capi.KIND_SCAN, n))
    x = torch.ones(n, dtype=torch.float32, device=dev())
    gb.set_debug(spin_limit_us=2000, drop_tile=3, workspace=ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        gb.inclusive(x, workspace=ws, compensated=True, algo="two_pass")
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 3 * LAUNCH_BOUND_S
    assert gb.device_status(ws) == _capi.ERR_TIMEOUT
    gb.set_debug(workspace=ws)
    y = gb.inclusive(x, workspace=ws, compensated=True, algo="two_pass")
    assert torch.equal(y, torch.arange(1, n + 1, device=dev(), dtype=torch.float32))
    assert gb.device_status(ws) == 0


def test_cuda_graph_segmented_replay():
    """Capture the segmented scan once, then replay it on new data written into
    the same input buffer; the epoch kept on the device makes each replay
    start from clean status words."""
    off = synth.segment_offsets(2000, max_log2=14, seed=7)
    n = int(off[-1])
    g = SegmentedScanGraph(n, off, torch.int32, exclusive=True)
    for rep in range(10):
        a = synth.uniform_i32(n, 4, seed=50 + rep)
        y = g.run(torch.from_numpy(a).to(dev())).cpu().numpy()
        assert np.array_equal(y, oracle.seg_scan_i32(a, off, True)), rep
    assert g.device_status() == 0


@pytest.mark.parametrize("algo", ["auto", "single_pass", "partitioned", "resident"])
def test_cuda_graph_plain_scan_replay(algo):
    n = (1 << 20) + 5
    x = torch.empty(n, dtype=torch.float32, device=dev())
    y = torch.empty_like(x)
    ws = gb.Workspace(gb.workspace_bytes(torch.float32, _capi.KIND_SCAN, n))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gb.inclusive(x.zero_(), out=y, workspace=ws, compensated=True, algo=algo)  # lazy init
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gb.inclusive(x, out=y, workspace=ws, compensated=True, algo=algo)
    for rep in range(10):
        a = synth.normal_f32(n, seed=rep)
        x.copy_(torch.from_numpy(a))
        graph.replay()
        torch.cuda.synchronize()
        err, _ = oracle.max_rel_err(y.cpu().numpy(), oracle.scan_f32_ref(a), oracle.abs_scan_f32(a))
        assert err <= 1e-6


# ---- autograd -------------------------------------------------------------------

def test_gradcheck_fp64():
    x = torch.randn(8, 64, dtype=torch.float64, device=dev(), requires_grad=True)
    for excl in (False, True):
        assert torch.autograd.gradcheck(lambda t: gb.cumsum(t, -1, excl), (x,), eps=1e-6,
                                        atol=1e-9, rtol=1e-7)
    y = torch.randn(6, 5, 7, dtype=torch.float64, device=dev(), requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: gb.cumsum(t, 1), (y,))


def test_finite_differences_fp32():
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(4, 300, generator=g).to(dev())
    w = torch.randn(4, 300, generator=g).to(dev())
    xr = x.clone().requires_grad_(True)
    (gb.cumsum(xr) * w).sum().backward()
    h = 1e-2
    for (r, c) in [(0, 0), (1, 17), (2, 150), (3, 299)]:
        xp, xm = x.clone(), x.clone()
        xp[r, c] += h
        xm[r, c] -= h
        fd = ((gb.cumsum(xp) * w).sum() - (gb.cumsum(xm) * w).sum()).item() / (2 * h)
        assert abs(fd - xr.grad[r, c].item()) <= 1e-3 * max(1.0, abs(fd)) + 2e-2


def test_backward_matches_oracle_and_forward_matches_cumsum():
    rows, cols = 64, 3000
    a = synth.normal_f32(rows * cols, seed=8).reshape(rows, cols)
    gnp = synth.normal_f32(rows * cols, seed=9).reshape(rows, cols)
    x = to_dev(a).requires_grad_(True)
    y = gb.cumsum(x, -1)
    y.backward(to_dev(gnp))
    off = np.arange(rows + 1, dtype=np.int64) * cols
    err, _ = oracle.max_rel_err(y.detach().cpu().numpy(),
                                oracle.seg_scan_f32_ref(a.reshape(-1), off).reshape(rows, cols),
                                oracle.seg_abs_scan_f32(a.reshape(-1), off).reshape(rows, cols))
    assert err <= 1e-5
    err, _ = oracle.max_rel_err(x.grad.cpu().numpy(), oracle.rows_suffix_f32_ref(gnp),
                                oracle.rows_suffix_abs_f32(gnp))
    assert err <= 1e-5
    # dim != -1 goes through a transpose
    x2 = to_dev(a).requires_grad_(True)
    y2 = gb.cumsum(x2, 0)
    y2.backward(to_dev(gnp))
    ref = oracle.rows_suffix_f32_ref(np.ascontiguousarray(gnp.T)).T
    err, _ = oracle.max_rel_err(x2.grad.cpu().numpy(), ref,
                                oracle.rows_suffix_abs_f32(np.ascontiguousarray(gnp.T)).T)
    assert err <= 1e-5
