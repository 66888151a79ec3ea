"""torch.autograd wrapper of the fp32 solve.

FWFunction.apply(W, recompute=False, options=None) -> (D, P) for W of shape
(n, n) or (B, n, n) (CUDA, float32, missing edges = +inf, zero diagonal).
Forward runs fw_solve (or one batched launch for B graphs); backward runs
fw_backward(_strided), which maps dL/dD to dL/dW through the predecessor trees.
With recompute=True only W is kept between the passes and the backward pass
re-runs the forward solve to get D and P again (memory for time, the usual
training trade-off when a batch of distance matrices does not fit).
"""
from __future__ import annotations

import torch

from . import (BatchedPlan, FW_F32, fw_backward_strided, fw_solve_ex, fw_sync_status, padded)


def _forward(W: torch.Tensor, options):
    if W.dtype != torch.float32 or not W.is_cuda:
        raise TypeError("FWFunction needs a CUDA float32 weight tensor")
    batched = W.dim() == 3
    Wb = W if batched else W.unsqueeze(0)
    B, n = Wb.shape[0], Wb.shape[1]
    ld = padded(n)
    Dbuf = torch.empty((B, n, ld), dtype=torch.float32, device=W.device)
    Pbuf = torch.empty((B, n, ld), dtype=torch.int32, device=W.device)
    D, P = Dbuf[:, :, :n], Pbuf[:, :, :n]
    D.copy_(Wb)
    if B == 1:
        fw_solve_ex(D[0], P[0], options)
    else:
        plan = BatchedPlan([n] * B, [ld] * B, FW_F32, options)
        plan.solve([D[b] for b in range(B)], [P[b] for b in range(B)])
        fw_sync_status()
        plan.close()
    fw_sync_status()
    return D, P


class FWFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W, recompute=False, options=None):
        D, P = _forward(W, options)
        ctx.batched = W.dim() == 3
        ctx.recompute = bool(recompute)
        ctx.options = options
        if ctx.recompute:
            ctx.save_for_backward(W)
        else:
            ctx.save_for_backward(D, P)
        Dout, Pout = (D, P) if ctx.batched else (D[0], P[0])
        ctx.mark_non_differentiable(Pout)
        return Dout, Pout

    @staticmethod
    def backward(ctx, gD, gP):
        if ctx.recompute:
            (W,) = ctx.saved_tensors
            D, P = _forward(W, ctx.options)
        else:
            D, P = ctx.saved_tensors
        B, n, ld = D.shape[0], D.shape[1], D.stride(1)
        g = torch.zeros((B, n, ld), dtype=torch.float32, device=D.device)
        g[:, :, :n] = gD if ctx.batched else gD.unsqueeze(0)
        gW = torch.empty((B, n, ld), dtype=torch.float32, device=D.device)
        fw_backward_strided(g[:, :, :n], D, P, gW[:, :, :n])
        out = gW[:, :, :n]
        return (out if ctx.batched else out[0]).contiguous(), None, None


def shortest_paths(W, recompute: bool = False, options=None):
    """Differentiable all-pairs shortest distances (and predecessors) of W."""
    return FWFunction.apply(W, recompute, options)
