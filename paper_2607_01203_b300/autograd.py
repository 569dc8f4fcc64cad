"""torch.autograd.Function around the certified bounds (argument marshalling only).

``LEBFunction.apply(handle, x_nom, u_nom, radii)`` returns ``(r_lo, r_hi)`` from ``leb_bounds``; its backward
calls ``leb_bounds_backward`` (the hand-written adjoint kernels) for d(bounds)/d(x~, u~, radii).
"""
from __future__ import annotations

import torch

from . import binding


class LEBFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, handle, x_nom, u_nom, radii):
        x, u, r = x_nom.contiguous(), u_nom.contiguous(), radii.contiguous()
        out = handle.bounds(x, u, radii=r, want_AB=False)
        ctx.handle = handle
        ctx.save_for_backward(x, u, r)
        return out["r_lo"].clone(), out["r_hi"].clone()

    @staticmethod
    def backward(ctx, g_lo, g_hi):
        x, u, r = ctx.saved_tensors
        if g_lo is None:
            g_lo = torch.zeros(x.shape[0], ctx.handle.n_x, device=x.device)
        if g_hi is None:
            g_hi = torch.zeros(x.shape[0], ctx.handle.n_x, device=x.device)
        gx, gu, gr, _ = ctx.handle.bounds_backward(x, u, r, g_lo.float(), g_hi.float())
        return None, gx, gu, gr


def leb_bounds(handle, x_nom, u_nom, radii):
    """Differentiable certified bounds (r_lo, r_hi) for box sets centred at the nominal."""
    return LEBFunction.apply(handle, x_nom, u_nom, radii)
