"""Benchmark: inclusive prefix sum of int32, n = 2^30, values uniform in
[0, 255] (seed 0), on one GB300.

One step = one scan of the whole 2^30-element array with the algorithm and
launch shape the autotuner picked for this GPU and size (the single-pass
chained scan with decoupled look-back at 2^30: one persistent launch per
step), tile load through carry add and store.  The metric is GB/s = (bytes read + bytes written) / device time,
with 8 * 2^30 bytes per step; inputs (4 GiB) and outputs are larger than the
129 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  Extra fields: the roofline of the timed
kernel against the measured HBM copy bandwidth; the single-pass decoupled
look-back kernel's own figure at the same size (single_pass_vs_copy); the
end-to-end number through the public API with host buffers, next to a
copy-only run of the same host-link schedule; SM clocks sampled during the
timed region; the CPU oracle timed on a bounded sample (cpu_baseline); and
side measurements of the other kernels (single-pass, two-pass, int64, fp32
plain and compensated, the small-input resident scan at int32 2^20 with the
L2 flushed, segmented, row-wise forward/backward, compaction, device copy) at
their own sizes.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --profile-case scan|seg_f32|compact_i32 ...   (profiler target)

Under torchrun (N > 1) every rank runs its own replica on its own GPU (the
scan does not shard here: replicas only); value = bytes of all ranks / the
slowest rank's time.  ``--impl reference`` times the CPU oracle on the host
cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_LOG2 = 30
N = 1 << N_LOG2
VALUE_RANGE = 256  # uniform integers in [0, 255]
BYTES_PER_STEP = 2 * 4 * N  # int32 read + write
METRIC = "scan GB/s (read+write bytes/device time) and % of HBM roofline; fp32 max rel err"
WORKLOAD = "int32 inclusive scan, n=2^30, uniform [0,255], seed 0"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-side", action="store_true", help="skip the side measurements")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--algo", choices=["auto", "single_pass", "two_pass", "partitioned", "resident"],
                    default="auto", help="scan algorithm of the timed step (auto: the tuned "
                    "fastest algorithm and variant for this GPU and size)")
    ap.add_argument("--n-log2", type=int, default=N_LOG2,
                    help="array size 2^k (profiling runs use a smaller case; the benchmark "
                         "workload is 2^30)")
    prof = ap.add_argument_group("profiler targets (no timing, no JSON line)")
    prof.add_argument("--profile-case", choices=["scan", "seg_f32", "compact_i32"],
                      help="launch one workload --reps times and exit: a target for ncu")
    prof.add_argument("--dtype", choices=["i32", "i64", "f32", "f32c"], default="i32",
                      help="scan case: element type (f32c = compensated fp32)")
    prof.add_argument("--n", type=int, default=None, help="scan case: element count (else 2^--n-log2)")
    prof.add_argument("--variant", type=int, default=None, help="scan and compact_i32 cases: launch shape (else tuned)")
    prof.add_argument("--reps", type=int, default=4, help="launches of the case")
    return ap.parse_args(argv)


# ---- distributed helpers (also used by the CPU tests with gloo) -------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(bytes_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job GB/s: the bytes every rank moved over the slowest rank's time."""
    return bytes_per_rank * world / seconds_max / 1e9


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---- clocks ------------------------------------------------------------------

def bind_to_gpu_cpus(gpu_index: int):
    """Binds the calling thread to the CPUs that NVML lists as local to the GPU,
    so that the pinned host buffers allocated next sit in the GPU's NUMA node
    (on a two-socket host, pages on the far socket cross one more link on
    every copy).  Read-only NVML queries; nothing about the GPU changes.
    Returns the CPUs, or None where NVML or the query is unavailable."""
    import ctypes
    try:
        nv = ctypes.CDLL("libnvidia-ml.so.1")
    except OSError:
        return None
    if nv.nvmlInit_v2() != 0:
        return None
    try:
        h = ctypes.c_void_p()
        if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(h)) != 0:
            return None
        words = ((os.cpu_count() or 64) + 63) // 64
        mask = (ctypes.c_ulong * words)()
        if nv.nvmlDeviceGetCpuAffinity(h, ctypes.c_uint(words), mask) != 0:
            return None
        allowed = os.sched_getaffinity(0)
        cpus = [64 * i + b for i in range(words) for b in range(64)
                if (mask[i] >> b) & 1 and 64 * i + b in allowed]
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return cpus
    except (OSError, AttributeError):
        return None
    finally:
        nv.nvmlShutdown()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.5)

    def stop(self) -> dict:
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ---- peaks -------------------------------------------------------------------

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def cuda_time_ms(fn, reps: int, flush=None) -> tuple[float, float, float]:
    """(median, min, mean) ms of fn over reps, CUDA events on the current
    stream; flush() runs between reps outside the timed interval.  Events tick
    in steps of about 2 us on GB300, so for microsecond kernels the mean of
    many reps resolves what the median cannot."""
    import torch
    s = torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times), min(times), statistics.mean(times)


# ---- CPU oracle baseline ------------------------------------------------------

def cpu_oracle_baseline(h_in_np, budget_s: float = 10.0) -> dict:
    """The oracle's sequential scan (single host thread) on the same input:
    whole passes over the 2^30-element array until about budget_s seconds."""
    import numpy as np
    import oracle
    a = h_in_np
    out = np.empty_like(a)
    lib = oracle._load()
    reps, t_total = 0, 0.0
    while t_total < budget_s and reps < 20:
        t0 = time.perf_counter()
        lib.oracle_scan_i32(a.ctypes.data, out.ctypes.data, a.size, 0)
        t_total += time.perf_counter() - t0
        reps += 1
    secs = t_total / reps
    return {"value": round(2 * 4 * a.size / secs / 1e9, 3), "unit": "GB/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{reps} full passes of the sequential oracle over the same 2^{N_LOG2} "
                      f"int32 input on one host thread ({secs * 1e3:.0f} ms per pass)"}


def run_reference(args):
    """--impl reference: the CPU oracle, timed on the host cores."""
    import numpy as np
    import oracle
    import synth
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    sample_log2 = 26  # each step: a 2^26-element prefix of the 2^30 workload
    m = 1 << sample_log2
    a = np.empty(m, dtype=np.int32)
    synth.uniform_i32_into(a.ctypes.data, m, VALUE_RANGE, seed=0)
    out = np.empty_like(a)
    lib = oracle._load()
    for _ in range(args.warmup):
        lib.oracle_scan_i32(a.ctypes.data, out.ctypes.data, m, 0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        lib.oracle_scan_i32(a.ctypes.data, out.ctypes.data, m, 0)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = 2 * 4 * m * args.steps / total / 1e9
    sample = (f"each step scans the first 2^{sample_log2} elements of the 2^{N_LOG2} int32 "
              f"workload with the sequential CPU oracle on one host thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "sample_n": m},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---- side measurements ----------------------------------------------------------

def side_measurements(dev, peak) -> dict:
    """Each other kernel at its own configuration, CUDA-event timed (median of
    reps).  Inputs > L2 except the [4096, 8192] row tensors (128 MiB), which
    are timed with an L2 flush (a 512 MiB write) between reps."""
    import numpy as np
    import torch
    import synth
    import paper_2312_14874_gb300 as gb
    from paper_2312_14874_gb300 import _capi
    from paper_2312_14874_gb300.graphs import SegmentedScanGraph

    res = {}

    def rec(name, nbytes, ms):
        res[name] = {"gbs": round(nbytes / (ms * 1e-3) / 1e9, 1), "ms": round(ms, 4),
                     "frac_of_hbm": round(nbytes / (ms * 1e-3) / 1e9 / peak, 3)}

    reps = 20
    # int32 2^30 variants of the headline: exclusive, two-pass, copy references
    x = torch.empty(N, dtype=torch.int32, device=dev)
    x.random_(0, VALUE_RANGE)
    y = torch.empty_like(x)
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_SCAN, N), dev)
    from paper_2312_14874_gb300 import autotune

    def pick(fam, n, algo):
        return autotune.choose(fam, fam[5:], n, algo)[1]

    rec("i32_2^30_exclusive", 8 * N, cuda_time_ms(lambda: gb.exclusive(x, out=y, workspace=ws), reps)[0])
    for algo in ("single_pass", "two_pass", "partitioned"):
        v = pick("scan_i32", N, algo)
        rec(f"i32_2^30_{algo}", 8 * N, cuda_time_ms(
            lambda: gb.inclusive(x, out=y, workspace=ws, algo=algo, variant=v), reps)[0])
    for op in ("max", "min"):
        rec(f"i32_2^30_running_{op}_partitioned", 8 * N, cuda_time_ms(
            lambda: gb.scan(x, out=y, op=op, algo="partitioned", variant=1, workspace=ws), reps)[0])
    # stream compaction, half kept: bytes = payload + flags read, kept written
    keep = torch.rand(N, device=dev) < 0.5
    kept = int(keep.sum().item())
    flags = keep.view(torch.uint8)
    rec("compact_i32_2^30_half_kept", 5 * N + 4 * kept, cuda_time_ms(
        lambda: gb.compact(x, flags, out=y, workspace=ws), reps)[0])
    del keep, flags
    rec("copy_torch_4GiB", 8 * N, cuda_time_ms(lambda: y.copy_(x), reps)[0])
    rec("copy_gbscan_4GiB", 8 * N, cuda_time_ms(lambda: gb.copy_(y, x), reps)[0])
    for algo in ("single_pass", "partitioned"):
        for v in range(gb.num_variants(torch.int32)):
            rec(f"i32_2^30_{algo}_variant{v}", 8 * N, cuda_time_ms(
                lambda: gb.inclusive(x, out=y, workspace=ws, algo=algo, variant=v), reps)[0])
    del x, y
    # int64 2^29
    n64 = 1 << 29
    x = torch.empty(n64, dtype=torch.int64, device=dev).random_(0, 1 << 32)
    y = torch.empty_like(x)
    for algo in ("single_pass", "two_pass", "partitioned"):
        v = pick("scan_i64", n64, algo)
        rec(f"i64_2^29_{algo}", 16 * n64, cuda_time_ms(
            lambda: gb.inclusive(x, out=y, workspace=ws, algo=algo, variant=v), reps)[0])
    del x, y
    # int32 2^20, U{0..15} (the small configuration: L2-sized, so the L2 is
    # flushed between reps and the time is reported in microseconds too)
    n1 = 1 << 20
    x1 = torch.randint(0, 16, (n1,), dtype=torch.int32, device=dev)
    y1 = torch.empty_like(x1)
    flush_small = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    med1, _, mean1 = cuda_time_ms(lambda: gb.inclusive(x1, out=y1, workspace=ws), 200,
                                  lambda: flush_small.fill_(1))
    rec("i32_2^20_flushed", 8 * n1, mean1)
    res["i32_2^20_flushed"]["us"] = round(mean1 * 1e3, 2)
    res["i32_2^20_flushed"]["us_median"] = round(med1 * 1e3, 2)
    res["i32_2^20_flushed"]["algo"] = "auto: " + ":".join(str(v) for v in autotune.choose("scan_i32", "i32", n1, "auto"))
    # the persistent single-pass kernel at the same size, for comparison
    v1 = pick("scan_i32", n1, "single_pass")
    mean_sp = cuda_time_ms(lambda: gb.inclusive(x1, out=y1, workspace=ws, algo="single_pass", variant=v1),
                           200, lambda: flush_small.fill_(1))[2]
    rec("i32_2^20_flushed_single_pass", 8 * n1, mean_sp)
    res["i32_2^20_flushed_single_pass"]["us"] = round(mean_sp * 1e3, 2)
    del x1, y1, flush_small
    # fp32 2^28, plain and compensated
    nf = 1 << 28
    x = torch.randn(nf, device=dev)
    y = torch.empty_like(x)
    for algo in ("single_pass", "two_pass", "partitioned"):
        v = pick("scan_f32", nf, algo)
        rec(f"f32_2^28_plain_{algo}", 8 * nf, cuda_time_ms(
            lambda: gb.inclusive(x, out=y, workspace=ws, algo=algo, variant=v), reps)[0])
        v = pick("scan_f32c", nf, algo)
        rec(f"f32_2^28_compensated_{algo}", 8 * nf, cuda_time_ms(
            lambda: gb.inclusive(x, out=y, workspace=ws, compensated=True, algo=algo, variant=v),
            reps)[0])
    # the algorithm AUTO runs for compensated fp32 at this size
    rec("f32_2^28_compensated_auto", 8 * nf, cuda_time_ms(
        lambda: gb.inclusive(x, out=y, workspace=ws, compensated=True), reps)[0])
    # fp32 max relative error of the tuned plain and compensated scans:
    # max_k |y_k - ref_k| / sum_{i<=k} |a_i|, with ref = torch.cumsum in
    # float64 on the GPU (its own error, about log2(n) * 2^-53 relative, is far
    # below what is measured; this run may not call the CPU oracle, which the
    # full-size tests compare against); on U[0,1) of the 2^-24 grid and N(0,1)
    errs = {}
    for dist, make in (("uniform", lambda: torch.randint(0, 1 << 24, (nf,), device=dev).float() * 2.0 ** -24),
                       ("normal", lambda: torch.randn(nf, device=dev))):
        x.copy_(make())
        ref = torch.cumsum(x.double(), 0)
        den = torch.cumsum(x.abs().double(), 0)
        for comp in (False, True):
            gb.inclusive(x, out=y, workspace=ws, compensated=comp)
            diff = (y.double() - ref).abs_()
            rel = torch.where(den > 0, diff / den.clamp_min(1e-300),
                              torch.where(diff == 0, torch.zeros_like(diff), torch.full_like(diff, float("inf"))))
            errs[f"{dist}_{'compensated' if comp else 'plain'}"] = float(rel.max().item())
            del diff, rel
        del ref, den
    res["fp32_max_rel_err"] = {"n": nf, "bounds": {"plain": 1e-5, "compensated": 1e-6},
                               "reference": "torch.cumsum of the input in float64 on the GPU", **errs}
    del x, y
    # segmented: 65,536 log-uniform segments in [1, 2^16], exclusive, CUDA graph
    off = synth.segment_offsets(65536, max_log2=16, seed=0)
    ns = int(off[-1])
    for dt in (torch.int32, torch.float32):
        g = SegmentedScanGraph(ns, off, dt, exclusive=True, device=dev)
        if dt == torch.int32:
            g.x.random_(0, 4)
        else:
            g.x.uniform_()
        key = 'i32' if dt == torch.int32 else 'f32'
        rec(f"seg_{key}_65536segs_exclusive_graph",
            8 * ns + 8 * (off.size), cuda_time_ms(g.replay, reps)[0])
        # the plain scan of the same elements (tuned algorithm), and how much
        # longer the segmented scan takes per byte
        yp = torch.empty_like(g.x)
        rec(f"plain_{key}_same_n_exclusive", 8 * ns, cuda_time_ms(
            lambda: gb.exclusive(g.x, out=yp, workspace=ws), reps)[0])
        res[f"seg_{key}_time_per_byte_vs_plain"] = round(
            res[f"plain_{key}_same_n_exclusive"]["gbs"] / res[f"seg_{key}_65536segs_exclusive_graph"]["gbs"], 3)
        del g, yp
    res["seg_total_n"] = ns
    # rows [4096, 8192] fp32: forward and backward, L2 flushed between reps
    rows, cols = 4096, 8192
    xr = torch.randn(rows, cols, device=dev)
    yr = torch.empty_like(xr)
    flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    flush = lambda: flush_buf.fill_(1)
    rec("rows_f32_4096x8192_forward", 8 * rows * cols, cuda_time_ms(
        lambda: gb.rows(xr, out=yr, workspace=ws), reps, flush)[0])
    rec("rows_f32_4096x8192_backward", 8 * rows * cols, cuda_time_ms(
        lambda: gb.backward(xr, out=yr, workspace=ws), reps, flush)[0])
    rec("plain_f32_2^25_flushed", 8 * rows * cols, cuda_time_ms(
        lambda: gb.inclusive(xr.view(-1), out=yr.view(-1), workspace=ws), reps, flush)[0])
    del xr, yr, flush_buf
    return res


# ---- profiler targets -------------------------------------------------------------

def profile_case(args) -> int:
    """One workload launched --reps times, for a profiler: every launch is the
    same; the first ones warm the caches and load the module, so a profiler
    skips them.  Inputs are seeded and synthetic; nothing is checked here (the
    test suite does that).

    scan         the plain inclusive scan of --dtype, 2^--n-log2 (or --n)
                 elements, U[0,1) for floats, with --algo and --variant (tuned
                 when not given)
    seg_f32      the exclusive segmented scan of 20,000 segments with lengths
                 log-uniform in [1, 2^16] (116,893,251 fp32 elements, U[0,1))
    compact_i32  stream compaction of 2^28 int32 elements with half kept, with
                 --variant (tuned when not given)
    """
    import torch
    import paper_2312_14874_gb300 as gb
    from paper_2312_14874_gb300 import _capi
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    if args.profile_case == "scan":
        dt = {"i32": torch.int32, "i64": torch.int64, "f32": torch.float32, "f32c": torch.float32}[args.dtype]
        n = args.n if args.n is not None else 1 << args.n_log2
        if dt.is_floating_point:
            x = torch.rand(n, device=dev, generator=g)
        else:
            x = torch.randint(0, 256, (n,), dtype=dt, device=dev, generator=g)
        y = torch.empty_like(x)
        ws = gb.Workspace(gb.workspace_bytes(dt, _capi.KIND_SCAN, n), dev)
        for _ in range(args.reps):
            gb.inclusive(x, out=y, workspace=ws, algo=args.algo, variant=args.variant,
                         compensated=args.dtype == "f32c")
        torch.cuda.synchronize(dev)
        print(f"scan {args.dtype}: n={n}, algo={args.algo}, variant={args.variant}, "
              f"launches={args.reps}, status={gb.device_status(ws, dev)}")
    elif args.profile_case == "seg_f32":
        import synth
        off = synth.segment_offsets(20000, max_log2=16, seed=0)
        n = int(off[-1])
        x = torch.rand(n, device=dev, generator=g)
        y = torch.empty_like(x)
        o = torch.from_numpy(off).to(dev)
        ws = gb.Workspace(gb.workspace_bytes(torch.float32, _capi.KIND_SEGMENTED, n, off.size - 1), dev)
        for _ in range(args.reps):
            gb.segmented(x, o, True, out=y, workspace=ws)
        torch.cuda.synchronize(dev)
        print(f"seg_f32: n={n}, segments={off.size - 1}, launches={args.reps}, "
              f"status={gb.device_status(ws, dev)}")
    else:
        n = 1 << 28
        x = torch.randint(0, 1 << 30, (n,), dtype=torch.int32, device=dev, generator=g)
        flags = (torch.rand(n, device=dev, generator=g) < 0.5).view(torch.uint8)
        y = torch.empty_like(x)
        ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_COMPACT, n), dev)
        count = None
        for _ in range(args.reps):
            _, count = gb.compact(x, flags, out=y, workspace=ws, variant=args.variant)
        torch.cuda.synchronize(dev)
        print(f"compact_i32: n={n}, variant={args.variant}, kept={int(count.item())}, launches={args.reps}, "
              f"status={gb.device_status(ws, dev)}")
    return 0


# ---- main ------------------------------------------------------------------------

def main(argv=None) -> int:
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return profile_case(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    import paper_2312_14874_gb300 as gb
    from paper_2312_14874_gb300 import _capi, autotune

    global N, BYTES_PER_STEP, WORKLOAD
    if args.n_log2 != N_LOG2:
        N = 1 << args.n_log2
        BYTES_PER_STEP = 2 * 4 * N
        WORKLOAD = WORKLOAD.replace(f"n=2^{N_LOG2}", f"n=2^{args.n_log2}")
    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    peak, peak_kind = measured_hbm_peak()

    # host input in pinned memory (also the source of the e2e copies)
    local_cpus = bind_to_gpu_cpus(dev.index if dev.index is not None else 0)
    h_in = torch.empty(N, dtype=torch.int32, pin_memory=True)
    synth.uniform_i32_into(h_in.data_ptr(), N, VALUE_RANGE, seed=0)
    x = h_in.to(dev)
    y = torch.empty_like(x)
    ws = gb.Workspace(gb.workspace_bytes(torch.int32, _capi.KIND_SCAN, N), dev)
    algo, variant = autotune.choose("scan_i32", "i32", N, args.algo)
    if algo == "auto":  # no tuned table: the library's own rule at this size, spelled out
        algo = "single_pass"
    launches_per_step = 3 if algo == "two_pass" else 1
    stream = torch.cuda.current_stream(dev)

    def step():
        gb.inclusive(x, out=y, workspace=ws, variant=variant, algo=algo)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    # sanity: the last prefix is the total (mod 2^32)
    total = int(x.sum(dtype=torch.int64).item()) % (1 << 32)
    last = int(y[-1].item()) % (1 << 32)
    if total != last:
        raise RuntimeError("scan result failed the last == total check")

    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(dev)
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    barrier(dev)
    clk = clocks.stop()
    dev_status = gb.device_status(ws, dev)  # 0: no bounded wait ran out
    total_ms = starts[0].elapsed_time(ends[-1])
    launch_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    avg_launch_ms = sum(launch_ms) / len(launch_ms)
    secs_max = max_over_ranks(total_ms / 1e3, dev)
    value = aggregate(BYTES_PER_STEP * args.steps, secs_max, world)
    ms_per_step = secs_max * 1e3 / args.steps
    achieved = BYTES_PER_STEP / (avg_launch_ms * 1e-3) / 1e9

    # the single-pass decoupled look-back kernel at the same size, next to a
    # device copy of the same bytes timed in the same run: the figure the
    # single-pass target (85% of copy bandwidth at int32 2^30) is stated on
    sp_variant = autotune.choose("scan_i32", "i32", N, "single_pass")[1]
    sp_ms = cuda_time_ms(lambda: gb.inclusive(x, out=y, workspace=ws, algo="single_pass",
                                              variant=sp_variant), 20)[0]
    cp_ms = cuda_time_ms(lambda: y.copy_(x), 20)[0]
    gb.inclusive(x, out=y, workspace=ws, algo="single_pass", variant=sp_variant)
    torch.cuda.synchronize(dev)
    if int(y[-1].item()) % (1 << 32) != total:
        raise RuntimeError("single-pass result failed the last == total check")
    sp_vs_copy = {"kernel": "single-pass chained scan with decoupled look-back (lb_scan_kernel)",
                  "variant": sp_variant, "ms": round(sp_ms, 4),
                  "gbs": round(BYTES_PER_STEP / (sp_ms * 1e-3) / 1e9, 1),
                  "copy_gbs_same_run": round(BYTES_PER_STEP / (cp_ms * 1e-3) / 1e9, 1),
                  "frac_of_copy": round(cp_ms / sp_ms, 4),
                  "frac_of_hbm": round(BYTES_PER_STEP / (sp_ms * 1e-3) / 1e9 / peak, 4),
                  "target_frac_of_copy": 0.85}

    # end to end through the C ABI with host buffers (scan_inclusive_i32_host):
    # pinned host input -> device -> scan -> pinned host output, every step,
    # uploads, scans and downloads of 64 MiB pieces overlapping
    e2e = None
    if not args.no_e2e:
        h_out = torch.empty(N, dtype=torch.int32, pin_memory=True)
        e2e_steps = 4

        def e2e_step():
            gb.inclusive_host(h_in, h_out, d_buf=x, workspace=ws)

        # the host link alone: the same pieces (64 MiB) uploaded into the same
        # device buffer and downloaded again, upload and download overlapping
        # on two streams as in the library's pipeline, no scan
        piece = 16 << 20
        s_dn = torch.cuda.Stream(dev)

        def link_step():
            for k0 in range(0, N, piece):
                k1 = min(N, k0 + piece)
                x[k0:k1].copy_(h_in[k0:k1], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(stream)
                s_dn.wait_event(ev)
                with torch.cuda.stream(s_dn):
                    h_out[k0:k1].copy_(x[k0:k1], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s_dn)
            stream.wait_event(ev)

        # The two alternate step by step, so that a burst of other traffic on
        # the host link (the host is shared) falls on both alike; each total
        # is the sum of its steps' event times.
        link_step()
        e2e_step()
        torch.cuda.synchronize(dev)
        if int(h_out[-1].item()) % (1 << 32) != total:
            raise RuntimeError("end-to-end result failed the last == total check")
        barrier(dev)
        e2e_ms = link_ms = 0.0
        for _ in range(e2e_steps):
            for fn, which in ((e2e_step, 0), (link_step, 1)):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                if which == 0:
                    e2e_ms += a.elapsed_time(b)
                else:
                    link_ms += a.elapsed_time(b)
        e2e_secs = max_over_ranks(e2e_ms / 1e3 / e2e_steps, dev)
        link_secs = max_over_ranks(link_ms / 1e3 / e2e_steps, dev)
        e2e = {"value": round(aggregate(BYTES_PER_STEP, e2e_secs, world), 3), "unit": "GB/s",
               "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": 4 * N,
               "ms_per_step": round(e2e_secs * 1e3, 3),
               "copy_only": {"value": round(aggregate(BYTES_PER_STEP, link_secs, world), 3), "unit": "GB/s",
                             "ms_per_step": round(link_secs * 1e3, 3),
                             "what": "the same 64 MiB pieces up and down through the same device buffer, "
                                     "upload and download overlapping on two streams, no scan"},
               "frac_of_copy_only": round(link_secs / e2e_secs, 4),
               "host_buffers": (f"pinned, allocated from {len(local_cpus)} CPUs local to the GPU (NVML)"
                                if local_cpus else "pinned")}
        del h_out

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.n_log2 == N_LOG2:
        cpu = cpu_oracle_baseline(h_in.numpy())

    side = None
    if rank == 0 and not args.no_side and args.n_log2 == N_LOG2:
        del y
        torch.cuda.empty_cache()
        side = side_measurements(dev, peak)

    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(prof) as f:
            tj = json.load(f)
        if (tj.get("kernel_variant") == variant and tj.get("algo") == algo
                and tj.get("source_stamp") == _source_stamp()):
            traffic = tj.get("bytes_per_launch_full")
    except (OSError, ValueError):
        pass

    if rank == 0:
        vinfo = gb.variant_info(torch.int32, _capi.KIND_SCAN, variant)
        if algo == "partitioned":
            # the partitioned kernel of a variant: its consumer warps, a loader
            # warp and a chunk scanner warp; at least three stages
            cw = vinfo["tile"] // (32 * vinfo["items"])
            vinfo = {"threads": (cw + 2) * 32, "items": vinfo["items"],
                     "stages": max(vinfo["stages"], 3), "tile": vinfo["tile"]}
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "dtype": "int32", "values": "uniform [0,255]",
                       "algo": algo, "variant": variant, **vinfo,
                       "l2": f"input and output {4 * N / 2**30:g} GiB each, larger than the 129 MB L2: no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy)",
                         "bytes_per_launch": BYTES_PER_STEP,
                         "avg_launch_ms": round(avg_launch_ms, 4)},
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "device_status": dev_status,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                       "reasons": clk["reasons"], "samples": clk["samples"],
                       "power_w_max": clk.get("power_w_max")},
            "single_pass_vs_copy": sp_vs_copy,
            "cpu_baseline": cpu,
            "elements_per_s": round(value * 1e9 / 8, 1),
            "side": side,
        }
        if side is not None:
            # the other parts of the metric: % of a device copy of the same
            # bytes measured in this run, and the fp32 errors
            line["frac_of_copy_today"] = round(value / side["copy_torch_4GiB"]["gbs"], 4)
            line["fp32_max_rel_err"] = side["fp32_max_rel_err"]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# The sources the timed int32 kernel (the single-pass look-back kernel, or the
# partitioned one when a tuned table picks it) is built and launched from:
# their templates and the tile code they use, the shared device definitions,
# the launcher, the int32 variant table, the host dispatch and the C header.
# The other kernels' sources (two-pass, resident, row-block, compaction) do
# not change their code.
STAMP_SOURCES = ("include/gbscan.h",
                 "paper_2312_14874_gb300/csrc/gbscan_device.cuh",
                 "paper_2312_14874_gb300/csrc/tile_common.cuh",
                 "paper_2312_14874_gb300/csrc/lookback.cuh",
                 "paper_2312_14874_gb300/csrc/partitioned.cuh",
                 "paper_2312_14874_gb300/csrc/gbscan_launch.cuh",
                 "paper_2312_14874_gb300/csrc/k_i32.cu",
                 "paper_2312_14874_gb300/csrc/capi.cu")


def _source_stamp() -> str:
    """Hash of the timed kernel's sources, to tell whether a recorded ncu
    traffic figure still describes the current kernel."""
    import hashlib
    h = hashlib.sha256()
    for rel in STAMP_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(rel.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
