"""CPU oracle for the prefix sum — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg (``bench.py --impl reference`` and the ``cpu_baseline`` field) may import
this package.  It shares no code with the CUDA library: the arithmetic lives
in ``oracle.c`` (plain sequential loops, one per definition, each citing the
paper) and is compiled by the host C compiler.

The numpy wrappers below only marshal arguments; the one piece of arithmetic
done here is the error metric of the float comparisons,
``max_k |y_k - ref_k| / sum_{i<=k} |a_i|`` (the denominator is itself an
oracle scan of |a|).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str | None = None, out: str | None = None,
          defines: tuple = ()) -> str:
    """Compile the oracle with gcc: -O2, no fast-math, no FMA contraction, so
    every operation rounds as written."""
    src = src or _SRC
    out = out or _LIB_PATH
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", *[f"-D{d}" for d in defines], src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _declare(lib):
    i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
    sig = {
        "oracle_scan_i32": [vp, vp, i64, ci],
        "oracle_scan_i64": [vp, vp, i64, ci],
        "oracle_scan_f32_ref": [vp, vp, i64, ci],
        "oracle_scan_f64_ref": [vp, vp, i64, ci],
        "oracle_scan_f32_plain_f64": [vp, vp, i64, ci],
        "oracle_abs_scan_f32": [vp, vp, i64, ci],
        "oracle_seg_scan_i32": [vp, vp, vp, i64, ci],
        "oracle_seg_scan_i64": [vp, vp, vp, i64, ci],
        "oracle_seg_scan_f32_ref": [vp, vp, vp, i64, ci],
        "oracle_seg_abs_scan_f32": [vp, vp, vp, i64, ci],
        "oracle_rows_suffix_f32_ref": [vp, vp, i64, i64, ci],
        "oracle_rows_suffix_f64_ref": [vp, vp, i64, i64, ci],
        "oracle_rows_suffix_abs_f32": [vp, vp, i64, i64, ci],
        "oracle_scan_max_i32": [vp, vp, i64, ci],
        "oracle_scan_min_i32": [vp, vp, i64, ci],
        "oracle_scan_max_f32": [vp, vp, i64, ci],
        "oracle_scan_min_f32": [vp, vp, i64, ci],
        "oracle_scan_max_i64": [vp, vp, i64, ci],
        "oracle_scan_min_i64": [vp, vp, i64, ci],
        "oracle_scan_max_u32": [vp, vp, i64, ci],
        "oracle_scan_min_u32": [vp, vp, i64, ci],
        "oracle_scan_u32": [vp, vp, i64, ci],
        "oracle_seg_scan_max_i32": [vp, vp, vp, i64, ci],
        "oracle_seg_scan_min_i32": [vp, vp, vp, i64, ci],
        "oracle_seg_scan_max_f32": [vp, vp, vp, i64, ci],
        "oracle_seg_scan_min_f32": [vp, vp, vp, i64, ci],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None
    lib.oracle_reduce_i32.argtypes = [vp, i64]
    lib.oracle_reduce_i32.restype = ctypes.c_int32
    lib.oracle_reduce_i64.argtypes = [vp, i64]
    lib.oracle_reduce_i64.restype = ctypes.c_int64
    lib.oracle_compact_u32.argtypes = [vp, vp, vp, i64]
    lib.oracle_compact_u32.restype = ctypes.c_int64
    return lib


def load_library(path: str):
    """Load an oracle shared object (used by the tests that plant mistakes in
    a separately compiled copy)."""
    return _declare(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


# ---- plain scans ----------------------------------------------------------

def scan_i32(a, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.int32)
    y = np.empty_like(a)
    (lib or _load()).oracle_scan_i32(a.ctypes.data, y.ctypes.data, a.size, int(exclusive))
    return y


def scan_i64(a, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.int64)
    y = np.empty_like(a)
    (lib or _load()).oracle_scan_i64(a.ctypes.data, y.ctypes.data, a.size, int(exclusive))
    return y


def scan_u32(a, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.uint32)
    y = np.empty_like(a)
    (lib or _load()).oracle_scan_u32(a.ctypes.data, y.ctypes.data, a.size, int(exclusive))
    return y


_OP_KINDS = {np.dtype(np.int32): "i32", np.dtype(np.float32): "f32",
             np.dtype(np.int64): "i64", np.dtype(np.uint32): "u32"}


def scan_op(a, op: str, exclusive: bool = False, lib=None) -> np.ndarray:
    """Running maximum or minimum (op "max" / "min") of int32, int64, uint32 or
    float32 input."""
    a = np.asarray(a)
    kind = _OP_KINDS.get(a.dtype)
    if kind is None or op not in ("max", "min"):
        raise TypeError("max / min scans take int32, int64, uint32 or float32")
    a = np.ascontiguousarray(a)
    y = np.empty_like(a)
    getattr(lib or _load(), f"oracle_scan_{op}_{kind}")(a.ctypes.data, y.ctypes.data, a.size,
                                                          int(exclusive))
    return y


def compact(a, flags, lib=None) -> np.ndarray:
    """The elements of a (4-byte dtype) whose flags are nonzero, in order."""
    a = np.ascontiguousarray(a)
    if a.dtype.itemsize != 4:
        raise TypeError("compaction moves 4-byte elements")
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    if f.size != a.size:
        raise ValueError("flags must match a in length")
    out = np.empty_like(a)
    k = (lib or _load()).oracle_compact_u32(a.ctypes.data, f.ctypes.data, out.ctypes.data, a.size)
    return out[:k]


def reduce_i32(a, lib=None) -> int:
    a = _c(a, np.int32)
    return int((lib or _load()).oracle_reduce_i32(a.ctypes.data, a.size))


def reduce_i64(a, lib=None) -> int:
    a = _c(a, np.int64)
    return int((lib or _load()).oracle_reduce_i64(a.ctypes.data, a.size))


def scan_f32_ref(a, exclusive: bool = False, lib=None) -> np.ndarray:
    """FP64 (compensated) prefix sums of float32 input."""
    a = _c(a, np.float32)
    y = np.empty(a.size, dtype=np.float64)
    (lib or _load()).oracle_scan_f32_ref(a.ctypes.data, y.ctypes.data, a.size, int(exclusive))
    return y


def scan_f64_ref(a, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.float64)
    y = np.empty(a.size, dtype=np.float64)
    (lib or _load()).oracle_scan_f64_ref(a.ctypes.data, y.ctypes.data, a.size, int(exclusive))
    return y


def scan_f32_plain_f64(a, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.float32)
    y = np.empty(a.size, dtype=np.float64)
    (lib or _load()).oracle_scan_f32_plain_f64(a.ctypes.data, y.ctypes.data, a.size,
                                               int(exclusive))
    return y


def abs_scan_f32(a, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.float32)
    y = np.empty(a.size, dtype=np.float64)
    (lib or _load()).oracle_abs_scan_f32(a.ctypes.data, y.ctypes.data, a.size, int(exclusive))
    return y


# ---- segmented scans ------------------------------------------------------

def _check_offsets(offsets, n):
    off = _c(offsets, np.int64)
    if off.size < 1 or off[0] != 0 or off[-1] != n or np.any(np.diff(off) < 0):
        raise ValueError("offsets must be monotone, start at 0 and end at n")
    return off


def seg_scan_i32(a, offsets, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.int32)
    off = _check_offsets(offsets, a.size)
    y = np.zeros_like(a)
    (lib or _load()).oracle_seg_scan_i32(a.ctypes.data, y.ctypes.data, off.ctypes.data,
                                         off.size - 1, int(exclusive))
    return y


def seg_scan_i64(a, offsets, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.int64)
    off = _check_offsets(offsets, a.size)
    y = np.zeros_like(a)
    (lib or _load()).oracle_seg_scan_i64(a.ctypes.data, y.ctypes.data, off.ctypes.data,
                                         off.size - 1, int(exclusive))
    return y


def seg_scan_op(a, offsets, op: str, exclusive: bool = False, lib=None) -> np.ndarray:
    """Segmented running maximum or minimum of int32 or float32 input: each
    segment on its own, an exclusive one starting from the operator's
    identity; elements outside the segments stay 0."""
    a = np.asarray(a)
    kind = {np.dtype(np.int32): "i32", np.dtype(np.float32): "f32"}.get(a.dtype)
    if kind is None or op not in ("max", "min"):
        raise TypeError("segmented max / min scans take int32 or float32")
    a = np.ascontiguousarray(a)
    off = _check_offsets(offsets, a.size)
    y = np.zeros_like(a)
    getattr(lib or _load(), f"oracle_seg_scan_{op}_{kind}")(a.ctypes.data, y.ctypes.data,
                                                             off.ctypes.data, off.size - 1,
                                                             int(exclusive))
    return y


def seg_scan_f32_ref(a, offsets, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.float32)
    off = _check_offsets(offsets, a.size)
    y = np.zeros(a.size, dtype=np.float64)
    (lib or _load()).oracle_seg_scan_f32_ref(a.ctypes.data, y.ctypes.data, off.ctypes.data,
                                             off.size - 1, int(exclusive))
    return y


def seg_abs_scan_f32(a, offsets, exclusive: bool = False, lib=None) -> np.ndarray:
    a = _c(a, np.float32)
    off = _check_offsets(offsets, a.size)
    y = np.zeros(a.size, dtype=np.float64)
    (lib or _load()).oracle_seg_abs_scan_f32(a.ctypes.data, y.ctypes.data, off.ctypes.data,
                                             off.size - 1, int(exclusive))
    return y


# ---- row-wise scans (forward cumsum along the last dim, and its gradient) --

def rows_scan_f32_ref(a2d, exclusive: bool = False, lib=None) -> np.ndarray:
    a2d = np.ascontiguousarray(a2d, dtype=np.float32)
    rows, cols = a2d.shape
    off = np.arange(rows + 1, dtype=np.int64) * cols
    return seg_scan_f32_ref(a2d.reshape(-1), off, exclusive, lib).reshape(rows, cols)


def rows_suffix_f32_ref(g2d, exclusive: bool = False, lib=None) -> np.ndarray:
    g2d = np.ascontiguousarray(g2d, dtype=np.float32)
    rows, cols = g2d.shape
    y = np.empty((rows, cols), dtype=np.float64)
    (lib or _load()).oracle_rows_suffix_f32_ref(g2d.ctypes.data, y.ctypes.data, rows, cols,
                                                int(exclusive))
    return y


def rows_suffix_f64_ref(g2d, exclusive: bool = False, lib=None) -> np.ndarray:
    g2d = np.ascontiguousarray(g2d, dtype=np.float64)
    rows, cols = g2d.shape
    y = np.empty((rows, cols), dtype=np.float64)
    (lib or _load()).oracle_rows_suffix_f64_ref(g2d.ctypes.data, y.ctypes.data, rows, cols,
                                                int(exclusive))
    return y


def rows_suffix_abs_f32(g2d, exclusive: bool = False, lib=None) -> np.ndarray:
    g2d = np.ascontiguousarray(g2d, dtype=np.float32)
    rows, cols = g2d.shape
    y = np.empty((rows, cols), dtype=np.float64)
    (lib or _load()).oracle_rows_suffix_abs_f32(g2d.ctypes.data, y.ctypes.data, rows, cols,
                                                int(exclusive))
    return y


# ---- the float error metric -----------------------------------------------

def max_rel_err(y, ref, den) -> tuple[float, int]:
    """max_k |y_k - ref_k| / den_k with den_k = sum of |a_i| over the terms of
    y_k.  Where den_k is 0 the output must be exactly 0 (an empty or all-zero
    prefix), and a nonzero difference there counts as an infinite error.
    Returns (error, index of the worst element)."""
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1)
    den = np.asarray(den, dtype=np.float64).reshape(-1)
    if y.size == 0:
        return 0.0, -1
    diff = np.abs(y - ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(den > 0, diff / np.where(den > 0, den, 1.0),
                       np.where(diff == 0, 0.0, np.inf))
    rel = np.where(np.isnan(rel), np.inf, rel)
    k = int(np.argmax(rel))
    return float(rel[k]), k
