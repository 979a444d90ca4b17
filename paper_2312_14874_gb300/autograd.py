"""Differentiable scan: torch.autograd.Function over the row-scan kernels.

Forward: y = scan of x along ``dim`` (inclusive, or exclusive with 0 first;
the Section 1 definition applied to every row).  The Jacobian of a row scan is
constant, dy_k/dx_i = [i <= k] (exclusive: [i < k]), so backward needs no
saved tensors: dx = J^T g is the reverse (suffix) scan of the incoming
gradient, dx_i = sum_{k >= i} g_k (exclusive: k > i), computed by the
hand-written reverse-scan kernel (``scan_backward_*``).
"""
from __future__ import annotations

import torch


class Cumsum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor, dim: int = -1, exclusive: bool = False):
        import paper_2312_14874_gb300 as gb
        if x.dtype not in (torch.float32, torch.float64):
            raise TypeError("cumsum takes float32 or float64")
        d = dim % x.dim() if x.dim() > 0 else 0
        ctx.dim = d
        ctx.exclusive = bool(exclusive)
        if x.dim() == 0:
            return x.clone() if not exclusive else torch.zeros_like(x)
        xm = x.movedim(d, -1).contiguous()
        y = gb.rows(xm, exclusive=bool(exclusive))
        return y.movedim(-1, d)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        import paper_2312_14874_gb300 as gb
        if g.dim() == 0:
            return (g.clone() if not ctx.exclusive else torch.zeros_like(g)), None, None
        gm = g.movedim(ctx.dim, -1).contiguous()
        dx = gb.backward(gm, exclusive=ctx.exclusive)
        return dx.movedim(-1, ctx.dim), None, None
