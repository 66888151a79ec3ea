"""torch.autograd wrapper of the fp32 solve.

FWFunction.apply(W, recompute=False, options=None) -> (D, P) for W of shape
(n, n) or (B, n, n) (CUDA, float32, missing edges = +inf, zero diagonal).
Forward runs fw_solve (or one batched launch for B graphs); backward runs
fw_backward(_strided), which maps dL/dD to dL/dW through the predecessor trees.
With recompute=True only W is kept between the passes and the backward pass
re-runs the forward solve to get D and P again (memory for time, the usual
training trade-off when a batch of distance matrices does not fit).

Batched plans are cached per (device, batch, n, options): a training step
reuses the plan's device tables and recorded CUDA graph (new output buffers
only refresh the plan's argument table), so the step allocates nothing in the
library.  When n is a multiple of 4 the tensors keep leading dimension n and
the gradients pass through without copies.
"""
from __future__ import annotations

import threading
from collections import OrderedDict

import torch

from . import (BatchedPlan, FW_F32, fw_backward_strided, fw_solve_ex, fw_sync_status, padded)

_PLANS: "OrderedDict[tuple, BatchedPlan]" = OrderedDict()
_PLANS_MAX = 8
_plans_lock = threading.Lock()


def _plan(device, B: int, n: int, ld: int, options) -> BatchedPlan:
    """The cached batched plan for B graphs of n vertices (created on first use)."""
    key = (device.index, B, n, ld, bytes(options) if options is not None else None)
    with _plans_lock:
        p = _PLANS.get(key)
        if p is not None:
            _PLANS.move_to_end(key)
            return p
        p = BatchedPlan([n] * B, [ld] * B, FW_F32, options)
        _PLANS[key] = p
        while len(_PLANS) > _PLANS_MAX:
            _PLANS.popitem(last=False)[1].close()
        return p


def clear_plan_cache() -> None:
    """Destroys every cached batched plan."""
    with _plans_lock:
        while _PLANS:
            _PLANS.popitem(last=False)[1].close()


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
        _plan(W.device, B, n, ld, options).solve([D[b] for b in range(B)],
                                                 [P[b] for b in range(B)])
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
        g = gD if ctx.batched else gD.unsqueeze(0)
        if g.stride() != D.stride():
            # the backward kernels take all four matrices with one layout
            gl = torch.zeros((B, n, ld), dtype=torch.float32, device=D.device)
            gl[:, :, :n] = g
            g = gl[:, :, :n]
        gW = torch.empty((B, n, ld), dtype=torch.float32, device=D.device)[:, :, :n]
        fw_backward_strided(g, D, P, gW)
        out = gW if ctx.batched else gW[0]
        return (out if ld == n else out.contiguous()), None, None


def shortest_paths(W, recompute: bool = False, options=None):
    """Differentiable all-pairs shortest distances (and predecessors) of W."""
    return FWFunction.apply(W, recompute, options)
