"""ctypes binding of the C ABI in ``include/gbscan.h`` (argument marshalling
only).  Every function here has the name and the argument order of the C entry
point it wraps; pointers and streams are passed as Python integers.

Loading fails loudly if the CUDA library cannot be built or loaded: there is
no fallback implementation of any entry point.
"""
from __future__ import annotations

import ctypes
import threading

from . import _build

_lock = threading.Lock()
_lib = None

# gbscan_status
OK, ERR_INVALID_ARG, ERR_ALIGNMENT, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {
    OK: "GBSCAN_OK", ERR_INVALID_ARG: "GBSCAN_ERR_INVALID_ARG",
    ERR_ALIGNMENT: "GBSCAN_ERR_ALIGNMENT", ERR_WORKSPACE: "GBSCAN_ERR_WORKSPACE",
    ERR_CUDA: "GBSCAN_ERR_CUDA", ERR_TIMEOUT: "GBSCAN_ERR_TIMEOUT",
    ERR_UNSUPPORTED: "GBSCAN_ERR_UNSUPPORTED",
}
# gbscan_algo
ALGO_AUTO, ALGO_SINGLE_PASS, ALGO_TWO_PASS, ALGO_PARTITIONED, ALGO_RESIDENT = 0, 1, 2, 3, 4
# gbscan_f32_mode
F32_PLAIN, F32_COMPENSATED = 0, 1
# gbscan_dtype
I32, I64, F32, F64, U32 = 0, 1, 2, 3, 4
# gbscan_kind
KIND_SCAN, KIND_SEGMENTED, KIND_ROWS, KIND_SCAN_MAX, KIND_SCAN_MIN, KIND_COMPACT = 0, 1, 2, 3, 4, 5
KIND_SEGMENTED_MAX, KIND_SEGMENTED_MIN = 6, 7
# gbscan_op
OP_SUM, OP_MAX, OP_MIN = 0, 1, 2

_vp, _i64, _i32, _u32, _sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                              ctypes.c_size_t)

# name -> argument types (all return gbscan_status unless listed in _RESTYPE)
_SIGNATURES = {
    "gbscan_workspace_size": [_i32, _i32, _i64, _i64, ctypes.POINTER(ctypes.c_size_t)],
    "gbscan_workspace_init": [_vp, _sz, _vp],
    "scan_inclusive_i32": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_exclusive_i32": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_inclusive_i64": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_exclusive_i64": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_inclusive_f32": [_vp, _vp, _i64, _i32, _vp, _sz, _i32, _i32, _vp],
    "scan_exclusive_f32": [_vp, _vp, _i64, _i32, _vp, _sz, _i32, _i32, _vp],
    "scan_inclusive_f64": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_exclusive_f64": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_segmented_batched_i32": [_vp, _vp, _i64, _vp, _i64, _i32, _vp, _sz, _i32, _vp],
    "scan_segmented_batched_f32": [_vp, _vp, _i64, _vp, _i64, _i32, _vp, _sz, _i32, _vp],
    "scan_rows_f32": [_vp, _vp, _i64, _i64, _i32, _vp, _sz, _i32, _vp],
    "scan_rows_f64": [_vp, _vp, _i64, _i64, _i32, _vp, _sz, _i32, _vp],
    "scan_backward_f32": [_vp, _vp, _i64, _i64, _i32, _vp, _sz, _i32, _vp],
    "scan_backward_f64": [_vp, _vp, _i64, _i64, _i32, _vp, _sz, _i32, _vp],
    "scan_get_device_status": [_vp, _vp],
    "gbscan_set_debug": [_vp, _sz, _u32, _i64, _u32, _vp],
    "gbscan_num_variants": [_i32, _i32],
    "gbscan_variant_info": [_i32, _i32, _i32] + [ctypes.POINTER(ctypes.c_int)] * 4,
    "gbscan_resident_max_n": [_i32, _i32, _i32, ctypes.POINTER(ctypes.c_int64)],
    "gbscan_copy": [_vp, _vp, _sz, _vp],
    "gbscan_status_string": [_i32],
    "gbscan_abi_version": [],
    "scan_inclusive_i32_noalloc": [_vp, _vp, _i64, _vp],
    "scan_op_i32": [_vp, _vp, _i64, _i32, _i32, _vp, _sz, _i32, _i32, _vp],
    "scan_op_f32": [_vp, _vp, _i64, _i32, _i32, _vp, _sz, _i32, _i32, _vp],
    "scan_op_i64": [_vp, _vp, _i64, _i32, _i32, _vp, _sz, _i32, _i32, _vp],
    "scan_op_u32": [_vp, _vp, _i64, _i32, _i32, _vp, _sz, _i32, _i32, _vp],
    "scan_inclusive_u32": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_exclusive_u32": [_vp, _vp, _i64, _vp, _sz, _i32, _i32, _vp],
    "scan_segmented_op_i32": [_vp, _vp, _i64, _vp, _i64, _i32, _i32, _vp, _sz, _i32, _vp],
    "scan_segmented_op_f32": [_vp, _vp, _i64, _vp, _i64, _i32, _i32, _vp, _sz, _i32, _vp],
    "compact_i32": [_vp, _vp, _vp, _i64, _vp, _vp, _sz, _i32, _vp],
    "compact_f32": [_vp, _vp, _vp, _i64, _vp, _vp, _sz, _i32, _vp],
    "scan_inclusive_i32_host": [_vp, _vp, _i64, _vp, _i64, _vp, _sz, _vp],
}
_RESTYPE = {"gbscan_status_string": ctypes.c_char_p, "gbscan_num_variants": ctypes.c_int,
            "gbscan_abi_version": ctypes.c_int}

ABI_VERSION = 2


def exported_names() -> list[str]:
    return list(_SIGNATURES)


def lib():
    """Build (if needed) and load libgbscan.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            h = ctypes.CDLL(path)
            for name, args in _SIGNATURES.items():
                f = getattr(h, name)
                f.argtypes = args
                f.restype = _RESTYPE.get(name, ctypes.c_int)
            if h.gbscan_abi_version() != ABI_VERSION:
                raise RuntimeError("libgbscan.so ABI version mismatch")
            _lib = h
    return _lib


def library_path() -> str:
    return _build.LIB


class GbscanError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().gbscan_status_string(status).decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({msg})")


def check(status: int, where: str) -> None:
    if status != OK:
        raise GbscanError(status, where)


def __getattr__(name):
    """Module-level access to the raw entry points, e.g. ``_capi.scan_inclusive_i32``."""
    if name in _SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
