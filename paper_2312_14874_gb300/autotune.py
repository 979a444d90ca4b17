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


def choose(kind_key: str, dtype_key: str, n: int) -> int:
    """Variant for a kernel family at size n: the tuned winner of the nearest
    size bucket at or above log2(n), else the largest bucket, else 0."""
    forced = os.environ.get("GBSCAN_VARIANT")
    if forced is not None:
        return int(forced)
    try:
        t = _table(gpu_key())
    except Exception:
        return 0
    entries = t.get(kind_key)
    if not entries:
        return 0
    b = max(0, math.ceil(math.log2(max(n, 1))))
    best = None
    for bucket, variant in sorted((int(k), int(v)) for k, v in entries.items()):
        best = variant
        if bucket >= b:
            return variant
    return best if best is not None else 0


def _time_ms(fn, reps: int = 10, warmup: int = 3) -> float:
    for _ in range(warmup):
        fn()
    stream = torch.cuda.current_stream()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(reps):
        start.record(stream)
        fn()
        end.record(stream)
        end.synchronize()
        times.append(start.elapsed_time(end))
    times.sort()
    return times[len(times) // 2]


def tune(sizes_log2=(20, 24, 28, 30), write: bool = True, families=None,
         verbose: bool = True) -> dict:
    """Time every variant of every family over the size ladder and record the
    fastest per (family, size bucket).  Inputs are zeros of each size (the
    kernels' cost does not depend on the values)."""
    import paper_2312_14874_gb300 as gb
    from . import _capi

    dev = torch.device("cuda", torch.cuda.current_device())
    free = torch.cuda.mem_get_info(dev)[0]
    plan = {
        "scan_i32": (torch.int32, _capi.KIND_SCAN, lambda x, y, v: gb.scan(x, out=y, variant=v)),
        "scan_i64": (torch.int64, _capi.KIND_SCAN, lambda x, y, v: gb.scan(x, out=y, variant=v)),
        "scan_f32": (torch.float32, _capi.KIND_SCAN, lambda x, y, v: gb.scan(x, out=y, variant=v)),
        "scan_f32c": (torch.float32, _capi.KIND_SCAN,
                      lambda x, y, v: gb.scan(x, out=y, variant=v, compensated=True)),
        "scan_f64": (torch.float64, _capi.KIND_SCAN, lambda x, y, v: gb.scan(x, out=y, variant=v)),
        "rows_f32": (torch.float32, _capi.KIND_ROWS,
                     lambda x, y, v: gb.rows(x.view(-1, 8192), out=y.view(-1, 8192), variant=v)),
        "bwd_f32": (torch.float32, _capi.KIND_ROWS,
                    lambda x, y, v: gb.backward(x.view(-1, 8192), out=y.view(-1, 8192), variant=v)),
    }
    if families:
        plan = {k: v for k, v in plan.items() if k in families}
    key = gpu_key(dev)
    result: dict = {}
    for fam, (dtype, kind, call) in plan.items():
        nv = gb.num_variants(dtype, kind)
        result[fam] = {}
        for lg in sizes_log2:
            n = 1 << lg
            esz = torch.empty((), dtype=dtype).element_size()
            if 2 * n * esz > 0.6 * free:
                continue
            x = torch.zeros(n, dtype=dtype, device=dev)
            y = torch.empty_like(x)
            times = [_time_ms(lambda: call(x, y, v)) for v in range(nv)]
            best = min(range(nv), key=lambda v: times[v])
            result[fam][str(lg)] = best
            if verbose:
                print(f"[tune] {fam} n=2^{lg}: " +
                      ", ".join(f"v{v}={t * 1e3:.1f}us" for v, t in enumerate(times)) +
                      f" -> v{best}", flush=True)
            del x, y
    if write:
        os.makedirs(TUNED_DIR, exist_ok=True)
        path = table_path(key)
        existing = {}
        try:
            with open(path) as f:
                existing = json.load(f)
        except (OSError, ValueError):
            pass
        existing.update(result)
        with open(path, "w") as f:
            json.dump(existing, f, indent=1, sort_keys=True)
        with _lock:
            _tables.pop(key, None)
    return result
