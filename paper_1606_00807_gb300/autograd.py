"""torch.autograd.Function around one analysis (argument marshalling only).

Forward: enkfmc_estimate -> enkfmc_assemble -> enkfmc_analyze on the tensors'
device and the current stream.  Backward: enkfmc_analyze_adjoint, which
returns dL/dX^b, dL/dy and dL/d diag(R); Z is treated as a constant input.
The handle keeps the forward's factors and increments, so a backward must
follow its own forward on that handle (checked with a generation counter).
"""
from __future__ import annotations

import torch

from . import binding as B


class EnKFMCAnalysis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Xb, y, R, Z, handle):
        h = handle
        h.set_stream(torch.cuda.current_stream(Xb.device).cuda_stream)
        Xb, y, R, Z = (t.contiguous() for t in (Xb, y, R, Z))
        T = torch.empty((Xb.shape[1], h.info.pmax), device=Xb.device, dtype=Xb.dtype)
        D = torch.empty(Xb.shape[1], device=Xb.device, dtype=Xb.dtype)
        Xa = torch.empty_like(Xb)
        h.estimate(Xb, T, D)
        h.assemble(Xb, T, D, R)
        h.analyze(Xb, y, R, Z, Xa)
        h.generation = getattr(h, "generation", 0) + 1
        ctx.h = h
        ctx.gen = h.generation
        ctx.save_for_backward(Xb, y, R, Z, T, D)
        return Xa

    @staticmethod
    def backward(ctx, Xa_bar):
        h = ctx.h
        if getattr(h, "generation", None) != ctx.gen:
            raise RuntimeError("the handle ran another analysis since this forward")
        Xb, y, R, Z, T, D = ctx.saved_tensors
        Xa_bar = Xa_bar.contiguous()
        Xb_bar = torch.empty_like(Xb)
        y_bar = torch.empty_like(y)
        R_bar = torch.empty_like(R)
        h.set_stream(torch.cuda.current_stream(Xb.device).cuda_stream)
        h.analyze_adjoint(Xa_bar, y_bar, R_bar, Xb_bar)
        return Xb_bar, y_bar, R_bar, None, None


def analysis(Xb, y, R, Z, handle):
    """X^a for member-major Xb [N][n] (differentiable in Xb, y and R)."""
    return EnKFMCAnalysis.apply(Xb, y, R, Z, handle)
