"""gbscan — prefix sums (scans) on GB300 (sm_103a).

The operation follows Zhang, Wang and Ross, "Parallel Prefix Sum with SIMD"
(ADMS'20), Section 1: the inclusive scan of [a_0, ..., a_{n-1}] under + is
[a_0, a_0 + a_1, ..., a_0 + ... + a_{n-1}]; the exclusive scan drops the last
prefix and starts with 0.  Every computation runs in the hand-written CUDA
kernels of ``libgbscan.so`` (C ABI in ``include/gbscan.h``); this module only
checks tensors, picks a workspace and a launch shape, and calls the C entry
points on the current torch stream.  There is no CPU fallback: a CPU tensor is
rejected.

Public API:
    inclusive(x), exclusive(x), scan(x, exclusive=...)  int32/int64/uint32/float32/float64
    scan(x, op="max" | "min")                           running max / min, int32/int64/uint32/float32
    compact(x, flags)                                    stream compaction, int32/float32
    inclusive_host(h_in)                                 int32 scan of a host array, pipelined
    segmented(x, offsets, exclusive=..., op=...)          CSR segments, int32/float32, sum/max/min
    rows(x, exclusive=...), backward(g, exclusive=...)    along the last dim, float32/float64
    cumsum(x, dim=-1, exclusive=False)                    differentiable (autograd)
    device_status(), copy_(dst, src), Workspace
    resident_max_n(dtype)                                the largest input algo="resident" takes

Algorithms (``algo=``): "auto" (the tuned table for this GPU, else the
library's rule: the resident scan where it fits, the single-pass scan above),
"single_pass" (chained scan with decoupled look-back), "two_pass" (reduce,
scan of the tile sums, scan with offsets), "partitioned" (Section 2.2's cache
partitioning with L2 as the cache) and "resident" (small inputs: one block
per tile, every tile held in shared memory).  ``variant`` picks the launch
shape (None: the tuned one).  The single-pass, partitioned and compaction
kernels prefetch their input into L2 about 12 MiB ahead of their copies
(environment variable GBSCAN_PREFETCH_BYTES; 1 turns it off).
"""
from __future__ import annotations

import threading

import torch

from . import _capi
from ._capi import GbscanError

__all__ = [
    "inclusive", "exclusive", "scan", "segmented", "rows", "backward", "cumsum",
    "device_status", "copy_", "Workspace", "workspace_bytes", "set_debug", "GbscanError",
    "num_variants", "variant_info", "resident_max_n", "compact", "inclusive_host",
]

_DTYPES = {
    torch.int32: (_capi.I32, "i32"),
    torch.int64: (_capi.I64, "i64"),
    torch.float32: (_capi.F32, "f32"),
    torch.float64: (_capi.F64, "f64"),
    torch.uint32: (_capi.U32, "u32"),
}
_ALGOS = {"auto": _capi.ALGO_AUTO, "single_pass": _capi.ALGO_SINGLE_PASS,
          "two_pass": _capi.ALGO_TWO_PASS, "partitioned": _capi.ALGO_PARTITIONED,
          "resident": _capi.ALGO_RESIDENT}


def _stream_handle(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def workspace_bytes(dtype: torch.dtype, kind: int, n: int, num_segments: int = 0) -> int:
    import ctypes
    out = ctypes.c_size_t(0)
    _capi.check(_capi.lib().gbscan_workspace_size(_DTYPES[dtype][0], kind, n, num_segments,
                                                  ctypes.byref(out)), "gbscan_workspace_size")
    return int(out.value)


class Workspace:
    """A zeroed device buffer for the scan status records.  One workspace may
    serve any sequence of calls on one stream; calls that can overlap in time
    need separate workspaces."""

    def __init__(self, nbytes: int, device=None):
        device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        nbytes = max(int(nbytes), 4096)
        self.buf = torch.zeros(nbytes, dtype=torch.uint8, device=device)
        self.nbytes = nbytes
        self.device = device

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()


_ws_lock = threading.Lock()
_ws_cache: dict[tuple[int, int], Workspace] = {}


def _workspace_for(device: torch.device, need: int) -> Workspace:
    key = (device.index, _stream_handle(device))
    with _ws_lock:
        ws = _ws_cache.get(key)
        if ws is None or ws.nbytes < need:
            grow = max(need, 2 * ws.nbytes if ws is not None else 0)
            ws = Workspace(grow, device)
            _ws_cache[key] = ws
    return ws


def _check_cuda(x: torch.Tensor, name: str):
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (gbscan has no CPU path)")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _variant(kind: str, dtype_key: str, n: int, variant) -> int:
    if variant is not None:
        return int(variant)
    from . import autotune
    return autotune.choose(kind, dtype_key, n)[1]


_OPS = {"sum": _capi.OP_SUM, "max": _capi.OP_MAX, "min": _capi.OP_MIN}


def scan(x: torch.Tensor, exclusive: bool = False, *, out: torch.Tensor | None = None,
         algo: str = "auto", compensated: bool = False, variant: int | None = None,
         workspace: Workspace | None = None, op: str = "sum") -> torch.Tensor:
    """Prefix sum (or, with ``op="max"`` / ``"min"``, running maximum / minimum
    of int32 and float32) of a contiguous CUDA tensor, flattened.  ``out`` may
    be ``x`` (in place).  ``compensated`` selects TwoSum-pair carries for
    float32 sums."""
    _check_cuda(x, "x")
    if x.dtype not in _DTYPES:
        raise TypeError(f"unsupported dtype {x.dtype}")
    code, key = _DTYPES[x.dtype]
    if out is None:
        out = torch.empty_like(x)
    else:
        _check_cuda(out, "out")
        if out.dtype != x.dtype or out.numel() != x.numel() or out.device != x.device:
            raise ValueError("out must match x in dtype, size and device")
    n = x.numel()
    if n == 0:
        return out
    if compensated and x.dtype != torch.float32:
        raise ValueError("compensated mode applies to float32")
    if op not in _OPS:
        raise ValueError(f"unknown op {op!r}")
    if op != "sum":
        if x.dtype not in (torch.int32, torch.int64, torch.uint32, torch.float32) or compensated:
            raise TypeError("max / min scans take int32, int64, uint32 or float32 (no compensation)")
        if algo not in _ALGOS:
            raise ValueError(f"unknown algo {algo!r}")
        v = 0 if variant is None else int(variant)
        ws = workspace or _workspace_for(x.device, workspace_bytes(x.dtype, _capi.KIND_SCAN, n))
        fn = getattr(_capi.lib(), f"scan_op_{key}")
        _capi.check(fn(x.data_ptr(), out.data_ptr(), n, _OPS[op], int(exclusive), ws.ptr, ws.nbytes,
                       _ALGOS[algo], v, _stream_handle(x.device)), "scan_op")
        return out
    if key == "u32":
        # uint32 sums are the int32 sums of the same bits (modulo 2^32): the
        # int32 tuning applies
        key_tune = "i32"
    else:
        key_tune = key
    kind_key = "scan_" + key_tune + ("c" if compensated else "")
    if algo not in _ALGOS:
        raise ValueError(f"unknown algo {algo!r}")
    if variant is None:
        from . import autotune
        algo, v = autotune.choose(kind_key, key_tune, n, algo)
    else:
        v = int(variant)
    ws = workspace or _workspace_for(x.device, workspace_bytes(x.dtype, _capi.KIND_SCAN, n))
    s = _stream_handle(x.device)
    L = _capi.lib()
    a = _ALGOS[algo]
    if key == "f32":
        fn = L.scan_exclusive_f32 if exclusive else L.scan_inclusive_f32
        mode = _capi.F32_COMPENSATED if compensated else _capi.F32_PLAIN
        st = fn(x.data_ptr(), out.data_ptr(), n, mode, ws.ptr, ws.nbytes, a, v, s)
    else:
        fn = getattr(L, f"scan_{'exclusive' if exclusive else 'inclusive'}_{key}")
        st = fn(x.data_ptr(), out.data_ptr(), n, ws.ptr, ws.nbytes, a, v, s)
    _capi.check(st, "scan")
    return out


def inclusive(x: torch.Tensor, **kw) -> torch.Tensor:
    return scan(x, False, **kw)


def exclusive(x: torch.Tensor, **kw) -> torch.Tensor:
    return scan(x, True, **kw)


def inclusive_host(h_in: torch.Tensor, h_out: torch.Tensor | None = None, *,
                   d_buf: torch.Tensor | None = None, device=None,
                   workspace: Workspace | None = None) -> torch.Tensor:
    """Inclusive int32 scan of a HOST tensor into a host tensor, pipelined
    through the GPU (uploads, scans and downloads of 64 MiB pieces overlap).
    ``d_buf`` is the device staging buffer (default: 4 pieces).  Asynchronous
    on the device's current stream: synchronise before reading ``h_out``."""
    if not isinstance(h_in, torch.Tensor) or h_in.is_cuda or h_in.dtype != torch.int32:
        raise TypeError("h_in must be an int32 CPU tensor")
    if not h_in.is_contiguous():
        raise ValueError("h_in must be contiguous")
    n = h_in.numel()
    device = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    if h_out is None:
        h_out = torch.empty(n, dtype=torch.int32, pin_memory=True)
    if h_out.is_cuda or h_out.dtype != torch.int32 or h_out.numel() != n or not h_out.is_contiguous():
        raise ValueError("h_out must be a contiguous int32 CPU tensor of h_in's length")
    if n == 0:
        return h_out
    piece = 16 << 20
    if d_buf is None:
        d_buf = torch.empty(min(n, 4 * piece), dtype=torch.int32, device=device)
    _check_cuda(d_buf, "d_buf")
    ws = workspace or _workspace_for(
        device, workspace_bytes(torch.int32, _capi.KIND_SCAN, min(n, piece)))
    _capi.check(_capi.lib().scan_inclusive_i32_host(h_in.data_ptr(), h_out.data_ptr(), n,
                                                     d_buf.data_ptr(), d_buf.numel(), ws.ptr,
                                                     ws.nbytes, _stream_handle(device)),
                "scan_inclusive_i32_host")
    return h_out


def compact(x: torch.Tensor, flags: torch.Tensor, *, out: torch.Tensor | None = None,
            variant: int | None = None, workspace: Workspace | None = None):
    """Stream compaction: the elements of ``x`` (int32 or float32, flattened)
    whose ``flags`` (uint8 or bool, same length) are nonzero, in order.  One
    launch (the scan of the flags fused with the gather).  Returns ``(out,
    count)``: ``out`` holds x.numel() elements of which the first ``count``
    (a 0-d int64 CUDA tensor, read it with ``.item()``) are the result.
    ``variant`` None takes the tuned launch shape for the size."""
    _check_cuda(x, "x")
    _check_cuda(flags, "flags")
    if x.dtype not in (torch.int32, torch.float32):
        raise TypeError("compaction takes int32 or float32 values")
    if flags.dtype == torch.bool:
        flags = flags.view(torch.uint8)
    if flags.dtype != torch.uint8 or flags.numel() != x.numel() or flags.device != x.device:
        raise ValueError("flags must be uint8 or bool of x's length, on x's device")
    n = x.numel()
    if out is None:
        out = torch.empty_like(x)
    else:
        _check_cuda(out, "out")
        if out.dtype != x.dtype or out.numel() < n or out.device != x.device:
            raise ValueError("out must match x in dtype and device and hold x.numel() elements")
    count = torch.empty((), dtype=torch.int64, device=x.device)
    variant = _variant("compact_" + _DTYPES[x.dtype][1], _DTYPES[x.dtype][1], n, variant)
    ws = workspace or _workspace_for(x.device, workspace_bytes(x.dtype, _capi.KIND_COMPACT, n))
    fn = _capi.lib().compact_i32 if x.dtype == torch.int32 else _capi.lib().compact_f32
    _capi.check(fn(x.data_ptr(), flags.data_ptr(), out.data_ptr(), n, count.data_ptr(), ws.ptr,
                   ws.nbytes, int(variant), _stream_handle(x.device)), "compact")
    return out, count


def segmented(x: torch.Tensor, offsets: torch.Tensor, exclusive: bool = False, *,
              out: torch.Tensor | None = None, variant: int | None = None,
              workspace: Workspace | None = None, op: str = "sum") -> torch.Tensor:
    """Scan of every segment [offsets[s], offsets[s+1]) of a flat tensor, in one
    persistent launch.  ``offsets`` is an int64 CUDA tensor of S+1 entries from 0
    to x.numel().  ``op`` "max" / "min" gives each segment's running maximum /
    minimum (an exclusive one starts every segment from the operator's
    identity).  Malformed offsets are reported by device_status()."""
    _check_cuda(x, "x")
    _check_cuda(offsets, "offsets")
    if x.dtype not in (torch.int32, torch.float32):
        raise TypeError("segmented scans take int32 or float32")
    if offsets.dtype != torch.int64:
        raise TypeError("offsets must be int64")
    key = _DTYPES[x.dtype][1]
    if out is None:
        out = torch.empty_like(x)
    else:
        _check_cuda(out, "out")
    n = x.numel()
    nseg = offsets.numel() - 1
    if n == 0:
        return out
    if nseg < 1:
        raise ValueError("offsets needs at least two entries")
    if op not in _OPS:
        raise ValueError(f"unknown op {op!r}")
    if op == "sum":
        v = _variant("seg_" + key, key, n, variant)
        ws = workspace or _workspace_for(
            x.device, workspace_bytes(x.dtype, _capi.KIND_SEGMENTED, n, nseg))
        fn = getattr(_capi.lib(), f"scan_segmented_batched_{key}")
        _capi.check(fn(x.data_ptr(), out.data_ptr(), n, offsets.data_ptr(), nseg, int(exclusive),
                       ws.ptr, ws.nbytes, v, _stream_handle(x.device)), "segmented")
        return out
    v = 0 if variant is None else int(variant)
    kind = _capi.KIND_SEGMENTED_MAX if op == "max" else _capi.KIND_SEGMENTED_MIN
    ws = workspace or _workspace_for(x.device, workspace_bytes(x.dtype, kind, n, nseg))
    fn = getattr(_capi.lib(), f"scan_segmented_op_{key}")
    _capi.check(fn(x.data_ptr(), out.data_ptr(), n, offsets.data_ptr(), nseg, _OPS[op],
                   int(exclusive), ws.ptr, ws.nbytes, v, _stream_handle(x.device)), "segmented_op")
    return out


def _rows_call(name: str, kind_key: str, x: torch.Tensor, exclusive: bool, out, variant,
               workspace) -> torch.Tensor:
    _check_cuda(x, "x")
    if x.dtype not in (torch.float32, torch.float64):
        raise TypeError("row scans take float32 or float64")
    key = _DTYPES[x.dtype][1]
    if out is None:
        out = torch.empty_like(x)
    else:
        _check_cuda(out, "out")
    if x.numel() == 0:
        return out
    cols = x.shape[-1] if x.dim() > 0 else 1
    rows_ = x.numel() // cols
    v = _variant(kind_key + "_" + key, key, x.numel(), variant)
    ws = workspace or _workspace_for(
        x.device, workspace_bytes(x.dtype, _capi.KIND_ROWS, x.numel()))
    fn = getattr(_capi.lib(), f"{name}_{key}")
    _capi.check(fn(x.data_ptr(), out.data_ptr(), rows_, cols, int(exclusive), ws.ptr,
                   ws.nbytes, v, _stream_handle(x.device)), name)
    return out


def rows(x: torch.Tensor, exclusive: bool = False, *, out=None, variant=None,
         workspace=None) -> torch.Tensor:
    """Scan along the last dim (torch.cumsum(x, -1)), one launch for all rows."""
    return _rows_call("scan_rows", "rows", x, exclusive, out, variant, workspace)


def backward(g: torch.Tensor, exclusive: bool = False, *, out=None, variant=None,
             workspace=None) -> torch.Tensor:
    """Gradient of rows(): reverse (suffix) scan of g along the last dim."""
    return _rows_call("scan_backward", "bwd", g, exclusive, out, variant, workspace)


def cumsum(x: torch.Tensor, dim: int = -1, exclusive: bool = False) -> torch.Tensor:
    """Differentiable scan along ``dim`` (float32/float64), with the
    hand-written reverse-scan kernel as its backward."""
    from .autograd import Cumsum
    return Cumsum.apply(x, dim, exclusive)


def device_status(workspace: Workspace | None = None, device=None) -> int:
    """Synchronise the current stream and return (and clear) the first
    device-side error recorded in the workspace (0 = none)."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    ws = workspace or _workspace_for(device, 0)
    return int(_capi.lib().scan_get_device_status(ws.ptr, _stream_handle(device)))


def set_debug(spin_limit_us: int = 0, drop_tile: int = -1, delay_ns_max: int = 0,
              workspace: Workspace | None = None, device=None) -> None:
    """Test hooks stored in the workspace header (see gbscan_set_debug)."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None \
        else torch.device(device)
    ws = workspace or _workspace_for(device, 0)
    _capi.check(_capi.lib().gbscan_set_debug(ws.ptr, ws.nbytes, spin_limit_us, drop_tile,
                                             delay_ns_max, _stream_handle(device)),
                "gbscan_set_debug")


def copy_(dst: torch.Tensor, src: torch.Tensor) -> torch.Tensor:
    """Device-to-device copy with the library's vectorised copy kernel (the
    bandwidth reference)."""
    _check_cuda(dst, "dst")
    _check_cuda(src, "src")
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nbytes:
        raise ValueError("size mismatch")
    _capi.check(_capi.lib().gbscan_copy(src.data_ptr(), dst.data_ptr(), nbytes,
                                        _stream_handle(src.device)), "gbscan_copy")
    return dst


def num_variants(dtype: torch.dtype, kind: int = _capi.KIND_SCAN) -> int:
    return int(_capi.lib().gbscan_num_variants(_DTYPES[dtype][0], kind))


def variant_info(dtype: torch.dtype, kind: int, variant: int) -> dict:
    import ctypes
    t, i, s, tile = (ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int())
    _capi.check(_capi.lib().gbscan_variant_info(_DTYPES[dtype][0], kind, variant,
                                                ctypes.byref(t), ctypes.byref(i),
                                                ctypes.byref(s), ctypes.byref(tile)),
                "gbscan_variant_info")
    return {"threads": t.value, "items": i.value, "stages": s.value, "tile": tile.value}


def resident_max_n(dtype: torch.dtype, kind: int = _capi.KIND_SCAN, compensated: bool = False) -> int:
    """The largest input that ``algo="resident"`` takes for this dtype and kind
    (plain scan, running max or min) on the current device."""
    import ctypes
    n = ctypes.c_int64(0)
    mode = _capi.F32_COMPENSATED if compensated else _capi.F32_PLAIN
    _capi.check(_capi.lib().gbscan_resident_max_n(_DTYPES[dtype][0], kind, mode, ctypes.byref(n)),
                "gbscan_resident_max_n")
    return n.value
