"""Seeded synthetic inputs (counter-based SplitMix64), shared by the oracle
side and the GPU side.

This module draws numbers only; it holds no prefix-sum arithmetic.  The
generator and the derived distributions are defined in ``synth.c``.  The
paper's workloads are "random data" (Section 4.1); the concrete shapes used
here (uniform small integers, uniform floats on the 2^-24 grid, standard
normals, log-uniform segment lengths) are the synthetic stand-ins.

Every function has two forms: one that returns a numpy array, and a ``*_into``
form that fills caller-owned host memory given as an integer address (for
example a pinned ``torch`` tensor's ``data_ptr()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` with the host C compiler (no GPU code)."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u64, i64, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
            lib.synth_raw_u64.argtypes = [u64, u64, vp, i64, i64]
            lib.synth_uniform_i32.argtypes = [u64, u64, u64, vp, i64]
            lib.synth_uniform_i64.argtypes = [u64, u64, u64, vp, i64]
            lib.synth_unit_f32.argtypes = [u64, u64, vp, i64]
            lib.synth_normal_f32.argtypes = [u64, u64, vp, i64]
            lib.synth_normal_f64.argtypes = [u64, u64, vp, i64]
            lib.synth_segment_offsets.argtypes = [u64, u64, i64, ctypes.c_int, vp]
            lib.synth_segment_offsets.restype = i64
            for f in (lib.synth_raw_u64, lib.synth_uniform_i32, lib.synth_uniform_i64,
                      lib.synth_unit_f32, lib.synth_normal_f32, lib.synth_normal_f64):
                f.restype = None
            _lib = lib
    return _lib


# ---- pointer forms --------------------------------------------------------

def raw_u64_into(ptr: int, n: int, seed: int = 0, stream: int = 0, first: int = 0) -> None:
    _load().synth_raw_u64(seed, stream, ptr, n, first)


def uniform_i32_into(ptr: int, n: int, m: int, seed: int = 0, stream: int = 0) -> None:
    if not 1 <= m <= 1 << 32:
        raise ValueError("m must be in [1, 2^32]")
    _load().synth_uniform_i32(seed, stream, m, ptr, n)


def uniform_i64_into(ptr: int, n: int, m: int, seed: int = 0, stream: int = 0) -> None:
    if not 1 <= m <= 1 << 32:
        raise ValueError("m must be in [1, 2^32]")
    _load().synth_uniform_i64(seed, stream, m, ptr, n)


def unit_f32_into(ptr: int, n: int, seed: int = 0, stream: int = 0) -> None:
    _load().synth_unit_f32(seed, stream, ptr, n)


def normal_f32_into(ptr: int, n: int, seed: int = 0, stream: int = 0) -> None:
    _load().synth_normal_f32(seed, stream, ptr, n)


def normal_f64_into(ptr: int, n: int, seed: int = 0, stream: int = 0) -> None:
    _load().synth_normal_f64(seed, stream, ptr, n)


# ---- numpy forms ----------------------------------------------------------

def raw_u64(n: int, seed: int = 0, stream: int = 0, first: int = 0) -> np.ndarray:
    a = np.empty(n, dtype=np.uint64)
    raw_u64_into(a.ctypes.data, n, seed, stream, first)
    return a


def uniform_i32(n: int, m: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    a = np.empty(n, dtype=np.int32)
    uniform_i32_into(a.ctypes.data, n, m, seed, stream)
    return a


def uniform_i64(n: int, m: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    a = np.empty(n, dtype=np.int64)
    uniform_i64_into(a.ctypes.data, n, m, seed, stream)
    return a


def unit_f32(n: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    a = np.empty(n, dtype=np.float32)
    unit_f32_into(a.ctypes.data, n, seed, stream)
    return a


def normal_f32(n: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    a = np.empty(n, dtype=np.float32)
    normal_f32_into(a.ctypes.data, n, seed, stream)
    return a


def normal_f64(n: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    a = np.empty(n, dtype=np.float64)
    normal_f64_into(a.ctypes.data, n, seed, stream)
    return a


def segment_offsets(num_segments: int, max_log2: int = 16, seed: int = 0,
                    stream: int = 0) -> np.ndarray:
    """CSR offsets (int64, num_segments + 1 entries) of log-uniform lengths in
    [1, 2^max_log2]."""
    off = np.empty(num_segments + 1, dtype=np.int64)
    _load().synth_segment_offsets(seed, stream, num_segments, max_log2, off.ctypes.data)
    return off
