"""Autotuner for the launch shape (threads per block, items per thread,
pipeline stages) of every kernel family.

The paper's lesson is that tuning knobs such as the dilation factor are hard
to set by hand and that partition sizes are best derived from the hardware
(Section 5, Observation 1).  Here the knobs are the tile shape and the depth of
the TMA pipeline; ``tune()`` times every variant of a family with CUDA events
on the current GPU, over a ladder of sizes, and writes the winners to a JSON
table keyed by the GPU name and SM count.  ``choose()`` reads that table (the
table shipped in ``tuned/`` or one written by ``tune()``) and falls back to
variant 0 for an unknown GPU or family.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
TUNED_DIR = os.path.join(_HERE, "tuned")
_lock = threading.Lock()
_tables: dict[str, dict] = {}


def gpu_key(device=None) -> str:
    d = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    props = torch.cuda.get_device_properties(d)
    name = "".join(c if c.isalnum() else "_" for c in props.name)
    return f"{name}_{props.multi_processor_count}sm"


def table_path(key: str) -> str:
    env = os.environ.get("GBSCAN_TUNE_FILE")
    return env if env else os.path.join(TUNED_DIR, key + ".json")


def _table(key: str) -> dict:
    with _lock:
        if key not in _tables:
            path = table_path(key)
            try:
                with open(path) as f:
                    _tables[key] = json.load(f)
            except (OSError, ValueError):
                _tables[key] = {}
        return _tables[key]


ALGOS = ("single_pass", "two_pass", "partitioned", "resident")
SINGLE_SHAPE_ALGOS = ("resident",)  # one launch shape: timed as variant 0 only


def _entry(kind_key: str, n: int):
    """The tuned entry of the nearest size bucket at or above log2(n), else of
    the largest bucket, else None."""
    try:
        t = _table(gpu_key())
    except Exception:
        return None
    entries = t.get(kind_key)
    if not entries:
        return None
    b = max(0, math.ceil(math.log2(max(n, 1))))
    best = None
    for bucket, entry in sorted(((int(k), v) for k, v in entries.items()), key=lambda kv: kv[0]):
        best = entry
        if bucket >= b:
            return entry
    return best


def choose(kind_key: str, dtype_key: str, n: int, algo: str = "auto") -> tuple[str, int]:
    """(algorithm, variant) for a kernel family at size n.  For plain scans a
    tuned entry holds the fastest variant of every algorithm and the fastest
    pair overall ("best"), which is what algo="auto" takes; other families
    have one algorithm and an entry is the variant.  Without a table: the
    requested algorithm (the library's own AUTO rule for "auto") and variant 0."""
    forced = os.environ.get("GBSCAN_VARIANT")
    if forced is not None:
        return algo, int(forced)
    entry = _entry(kind_key, n)
    if entry is None:
        return algo, 0
    if isinstance(entry, dict):
        if algo == "auto":
            a, v = entry["best"].split(":")
            return a, int(v)
        return algo, int(entry.get(algo, 0))
    return algo, int(entry)


_flush_buf: torch.Tensor | None = None


def _time_ms(fn, reps: int = 10, warmup: int = 3) -> float:
    """Device time of fn (CUDA events, trimmed mean).  Before each rep a 256 MiB fill
    keeps the GPU busy while the host enqueues fn (so the host's enqueue time
    is not timed, which at small sizes would dwarf the kernel) and evicts the
    input from L2, as the benchmark does."""
    global _flush_buf
    if _flush_buf is None:
        _flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=torch.cuda.current_device())
    for _ in range(warmup):
        fn()
    stream = torch.cuda.current_stream()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(reps):
        _flush_buf.fill_(1)
        start.record(stream)
        fn()
        end.record(stream)
        end.synchronize()
        times.append(start.elapsed_time(end))
    # events tick in steps of about 2 us on GB300: a trimmed mean resolves
    # finer differences than the median between small kernels
    times.sort()
    k = len(times) // 10
    kept = times[k:len(times) - k] or times
    return sum(kept) / len(kept)


def tune(sizes_log2=(20, 22, 24, 26, 28, 30), write: bool = True, families=None,
         verbose: bool = True) -> dict:
    """Time every variant of every family over the size ladder and record the
    fastest per (family, size bucket); for plain scans, every variant of every
    algorithm.  Inputs are zeros of each size (the kernels' cost does not
    depend on the values)."""
    import paper_2312_14874_gb300 as gb
    from . import _capi

    dev = torch.device("cuda", torch.cuda.current_device())
    free = torch.cuda.mem_get_info(dev)[0]
    plain = {
        "scan_i32": (torch.int32, False),
        "scan_i64": (torch.int64, False),
        "scan_f32": (torch.float32, False),
        "scan_f32c": (torch.float32, True),
        "scan_f64": (torch.float64, False),
    }
    rowwise = {
        "rows_f32": (torch.float32, lambda x, y, v: gb.rows(x.view(-1, 8192), out=y.view(-1, 8192), variant=v)),
        "bwd_f32": (torch.float32, lambda x, y, v: gb.backward(x.view(-1, 8192), out=y.view(-1, 8192),
                                                                variant=v)),
    }
    segmented = {"seg_i32": torch.int32, "seg_f32": torch.float32}
    compaction = {"compact_i32": torch.int32, "compact_f32": torch.float32}
    if families:
        plain = {k: v for k, v in plain.items() if k in families}
        rowwise = {k: v for k, v in rowwise.items() if k in families}
        segmented = {k: v for k, v in segmented.items() if k in families}
        compaction = {k: v for k, v in compaction.items() if k in families}
    key = gpu_key(dev)
    result: dict = {}

    def sizes(dtype):
        esz = torch.empty((), dtype=dtype).element_size()
        for lg in sizes_log2:
            if 2 * (1 << lg) * esz <= 0.6 * free:
                yield lg

    for fam, (dtype, comp) in plain.items():
        result[fam] = {}
        nv = gb.num_variants(dtype, _capi.KIND_SCAN)
        for lg in sizes(dtype):
            x = torch.zeros(1 << lg, dtype=dtype, device=dev)
            y = torch.empty_like(x)
            entry, best_t = {}, None
            for algo in ALGOS:
                if algo == "resident" and (1 << lg) > gb.resident_max_n(dtype, compensated=comp):
                    continue
                nva = 1 if algo in SINGLE_SHAPE_ALGOS else nv
                times = [_time_ms(lambda: gb.scan(x, out=y, algo=algo, variant=v, compensated=comp))
                         for v in range(nva)]
                v = min(range(nva), key=lambda i: times[i])
                entry[algo] = v
                if best_t is None or times[v] < best_t:
                    best_t, entry["best"] = times[v], f"{algo}:{v}"
                if verbose:
                    print(f"[tune] {fam} n=2^{lg} {algo}: " +
                          ", ".join(f"v{i}={t * 1e3:.1f}us" for i, t in enumerate(times)), flush=True)
            result[fam][str(lg)] = entry
            if verbose:
                print(f"[tune] {fam} n=2^{lg} -> {entry['best']}", flush=True)
            del x, y
    for fam, (dtype, call) in rowwise.items():
        result[fam] = {}
        nv = gb.num_variants(dtype, _capi.KIND_ROWS)
        for lg in sizes(dtype):
            if lg < 13:
                continue
            x = torch.zeros(1 << lg, dtype=dtype, device=dev)
            y = torch.empty_like(x)
            times = [_time_ms(lambda: call(x, y, v)) for v in range(nv)]
            best = min(range(nv), key=lambda v: times[v])
            result[fam][str(lg)] = best
            if verbose:
                print(f"[tune] {fam} n=2^{lg}: " +
                      ", ".join(f"v{v}={t * 1e3:.1f}us" for v, t in enumerate(times)) +
                      f" -> v{best}", flush=True)
            del x, y
    for fam, dtype in segmented.items():
        # segments with lengths log-uniform in [1, 2^16] (mean about 5900),
        # as many as fill about 2^lg elements
        import synth
        result[fam] = {}
        nv = gb.num_variants(dtype, _capi.KIND_SEGMENTED)
        for lg in sizes(dtype):
            if lg < 20:
                continue
            off = synth.segment_offsets(max(1, (1 << lg) // 5908), max_log2=16, seed=0)
            n = int(off[-1])
            o = torch.from_numpy(off).to(dev)
            x = torch.zeros(n, dtype=dtype, device=dev)
            y = torch.empty_like(x)
            times = [_time_ms(lambda: gb.segmented(x, o, exclusive=True, out=y, variant=v))
                     for v in range(nv)]
            best = min(range(nv), key=lambda v: times[v])
            bucket = max(0, math.ceil(math.log2(n)))
            result[fam][str(bucket)] = best
            if verbose:
                print(f"[tune] {fam} n={n}: " +
                      ", ".join(f"v{v}={t * 1e3:.1f}us" for v, t in enumerate(times)) +
                      f" -> v{best}", flush=True)
            del x, y, o
    for fam, dtype in compaction.items():
        # half the elements kept, at random
        result[fam] = {}
        nv = gb.num_variants(dtype, _capi.KIND_COMPACT)
        for lg in sizes(dtype):
            if lg < 20:
                continue
            x = torch.zeros(1 << lg, dtype=dtype, device=dev)
            y = torch.empty_like(x)
            g = torch.Generator(device=dev)
            g.manual_seed(0)
            f = (torch.rand(1 << lg, device=dev, generator=g) < 0.5).to(torch.uint8)
            times = [_time_ms(lambda: gb.compact(x, f, out=y, variant=v)) for v in range(nv)]
            best = min(range(nv), key=lambda v: times[v])
            result[fam][str(lg)] = best
            if verbose:
                print(f"[tune] {fam} n=2^{lg}: " +
                      ", ".join(f"v{v}={t * 1e3:.1f}us" for v, t in enumerate(times)) +
                      f" -> v{best}", flush=True)
            del x, y, f
    if write:
        os.makedirs(TUNED_DIR, exist_ok=True)
        path = table_path(key)
        existing = {}
        try:
            with open(path) as f:
                existing = json.load(f)
        except (OSError, ValueError):
            pass
        for fam, entries in result.items():  # merge by size bucket
            existing.setdefault(fam, {}).update(entries)
        with open(path, "w") as f:
            json.dump(existing, f, indent=1, sort_keys=True)
        with _lock:
            _tables.pop(key, None)
    return result
