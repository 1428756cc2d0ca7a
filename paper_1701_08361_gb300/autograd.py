"""torch.autograd.Function wrappers of the NLINV frame.

Forward runs nlinv_frame / nlinv_batch; backward runs nlinv_frame_vjp /
nlinv_batch_vjp, the hand-written reverse pass through the unrolled IRGNM /
CG (Sec. 2.2, Eqs. 2-5): one forward sweep records every Newton step's CG
in device memory, the reverse sweep reads it (the frames of a batch on their
own streams).  Differentiable inputs: the
gridded data Y (complex64), alpha_0 (0-d float64 tensor) and x_prev.
Gradients follow torch's complex convention (dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch

from . import nlinv as L


def _check_sync(plan):
    rc = L.nlinv_sync(plan)
    if rc != 0:
        raise L.NlinvError(rc, "device")


class NLINVFrame(torch.autograd.Function):
    """x^_M = NLINV(Y, alpha_0, x_prev) for one frame of `plan`."""

    @staticmethod
    def forward(ctx, Y, alpha0, x_prev, plan, turn):
        a0 = float(alpha0)
        L.nlinv_set_alpha0(plan, a0)
        x = torch.empty(plan.nx, dtype=torch.complex64, device=Y.device)
        L.nlinv_frame(plan, Y, turn, x_prev, x)
        _check_sync(plan)
        ctx.plan, ctx.turn, ctx.a0 = plan, turn, a0
        ctx.has_prev = x_prev is not None
        ctx.save_for_backward(Y, x_prev if x_prev is not None else Y.new_empty(0))
        return x

    @staticmethod
    def backward(ctx, gx):
        Y, xp = ctx.saved_tensors
        plan = ctx.plan
        L.nlinv_set_alpha0(plan, ctx.a0)
        Ybar = torch.empty_like(Y)
        xpb = torch.empty(plan.nx, dtype=torch.complex64, device=Y.device) if ctx.has_prev else None
        a0bar = L.nlinv_frame_vjp(plan, Y, ctx.turn, xp if ctx.has_prev else None, gx.contiguous(),
                                  Ybar, xpb)
        ga = torch.tensor(a0bar, dtype=torch.float64, device=Y.device)
        return Ybar, ga, xpb, None, None


def nlinv_frame(Y, alpha0, plan, turn=0, x_prev=None):
    """Differentiable single frame: returns x^_M (complex64 [n_x])."""
    return NLINVFrame.apply(Y, alpha0, x_prev, plan, turn)


class NLINVBatch(torch.autograd.Function):
    """Independent frames of one plan reconstructed together (nlinv_batch);
    Ys: [B, J*G*G] complex64, x_prevs: [B, n_x] or None."""

    @staticmethod
    def forward(ctx, Ys, alpha0, x_prevs, plan, turns):
        a0 = float(alpha0)
        L.nlinv_set_alpha0(plan, a0)
        B = Ys.shape[0]
        xs = torch.empty((B, plan.nx), dtype=torch.complex64, device=Ys.device)
        L.nlinv_batch([dict(plan=plan, Y=Ys[b], turn=turns[b],
                            x_prev=None if x_prevs is None else x_prevs[b], x_out=xs[b])
                       for b in range(B)])
        _check_sync(plan)
        ctx.plan, ctx.turns, ctx.a0 = plan, list(turns), a0
        ctx.has_prev = x_prevs is not None
        ctx.save_for_backward(Ys, x_prevs if x_prevs is not None else Ys.new_empty(0))
        return xs

    @staticmethod
    def backward(ctx, gxs):
        Ys, xps = ctx.saved_tensors
        plan = ctx.plan
        L.nlinv_set_alpha0(plan, ctx.a0)
        Ybar = torch.empty_like(Ys)
        xpb = torch.empty_like(xps) if ctx.has_prev else None
        gxs = gxs.contiguous()
        B = Ys.shape[0]
        a0 = L.nlinv_batch_vjp(plan, [Ys[b] for b in range(B)], ctx.turns,
                               [xps[b] for b in range(B)] if ctx.has_prev else None,
                               [gxs[b] for b in range(B)], [Ybar[b] for b in range(B)],
                               [xpb[b] for b in range(B)] if ctx.has_prev else None)
        ga = torch.tensor(sum(a0), dtype=torch.float64, device=Ys.device)
        return Ybar, ga, xpb, None, None


def nlinv_batch(Ys, alpha0, plan, turns, x_prevs=None):
    """Differentiable batch of independent frames: returns [B, n_x]."""
    return NLINVBatch.apply(Ys, alpha0, x_prevs, plan, turns)
