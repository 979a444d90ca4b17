"""CUDA-graph helpers: capture a scan once, replay it on new data.

A captured call needs no host synchronisation and allocates nothing: the
workspace is preallocated, and the launch epoch and tile counter live in the
workspace header on the device, so every replay starts from valid state.
"""
from __future__ import annotations

import numpy as np
import torch

import paper_2312_14874_gb300 as gb
from . import _capi


class SegmentedScanGraph:
    """The batched segmented scan of a fixed segment layout, captured in a CUDA
    graph.  ``run(x)`` copies x into the captured input buffer, replays the
    graph on the current stream and returns the output buffer."""

    def __init__(self, n: int, offsets, dtype: torch.dtype = torch.int32,
                 exclusive: bool = False, device=None, variant: int | None = None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        if isinstance(offsets, np.ndarray):
            offsets = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64))
        self.offsets = offsets.to(self.device, torch.int64).contiguous()
        nseg = self.offsets.numel() - 1
        self.x = torch.zeros(n, dtype=dtype, device=self.device)
        self.y = torch.empty_like(self.x)
        self.ws = gb.Workspace(gb.workspace_bytes(dtype, _capi.KIND_SEGMENTED, n, nseg),
                               self.device)
        self.exclusive = exclusive
        self.variant = variant
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self._call()  # first call outside capture: kernel attributes, occupancy
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._call()

    def _call(self):
        gb.segmented(self.x, self.offsets, exclusive=self.exclusive, out=self.y,
                     variant=self.variant, workspace=self.ws)

    def replay(self) -> torch.Tensor:
        self.graph.replay()
        return self.y

    def run(self, x: torch.Tensor) -> torch.Tensor:
        self.x.copy_(x, non_blocking=True)
        return self.replay()

    def device_status(self) -> int:
        return gb.device_status(self.ws, self.device)
