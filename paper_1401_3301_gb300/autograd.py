"""torch.autograd wrappers of the stiffness assembly and its backward kernels.

``StiffnessValues.apply(w, q, pattern, prec)`` returns the CSR values of the
stiffness matrix S(w, q) (Eq. stiffelemmat of the paper, P0 coefficient w) and
back-propagates any loss of them through ``fe_assemble_stiff_vjp``.

``StiffnessBilinear.apply(w, q, u, v, pattern, prec)`` returns L = u^T S(w, q) v
without forming the matrix; one call of ``fe_assemble_stiff_backward`` gives L,
dL/dw and dL/dq together, and the backward pass only scales them. u and v are
treated as constants.
"""
from __future__ import annotations

import torch

from . import fe


def _w_args(w):
    return (None, fe.COEF_NONE) if w is None else (w, fe.COEF_P0)


class StiffnessValues(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, q, pattern, prec):
        wt, kind = _w_args(w)
        vals = fe.fe_assemble_stiff(pattern, q, wt, kind, prec=prec)
        ctx.pattern, ctx.prec, ctx.kind = pattern, prec, kind
        ctx.has_w = w is not None
        ctx.save_for_backward(*([w, q] if w is not None else [q]))
        return vals

    @staticmethod
    def backward(ctx, grad_vals):
        saved = ctx.saved_tensors
        w, q = (saved[0], saved[1]) if ctx.has_w else (None, saved[0])
        T = torch.float32 if ctx.prec == fe.F32 else torch.float64
        p = ctx.pattern
        dw = torch.empty(p.nme, dtype=T, device=q.device) if (ctx.has_w and ctx.needs_input_grad[0]) else None
        dq = torch.empty((p.d, p.nq), dtype=T, device=q.device) if ctx.needs_input_grad[1] else None
        if dw is not None or dq is not None:
            fe.fe_assemble_stiff_vjp(p, q, w, ctx.kind, grad_vals.contiguous().to(T), dw, dq, prec=ctx.prec)
        return dw, (dq.to(q.dtype) if dq is not None else None), None, None


class StiffnessBilinear(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, q, u, v, pattern, prec):
        T = torch.float32 if prec == fe.F32 else torch.float64
        wt, kind = _w_args(w)
        L = torch.empty(1, dtype=T, device=q.device)
        dw = torch.empty(pattern.nme, dtype=T, device=q.device) if w is not None else None
        dq = torch.empty((pattern.d, pattern.nq), dtype=T, device=q.device)
        fe.fe_assemble_stiff_backward(pattern, q, wt, kind, u.contiguous().to(T), v.contiguous().to(T),
                                      L, dw, dq, prec=prec)
        ctx.save_for_backward(*([dw, dq] if dw is not None else [dq]))
        ctx.has_w = w is not None
        ctx.q_dtype = q.dtype
        return L[0]

    @staticmethod
    def backward(ctx, gL):
        saved = ctx.saved_tensors
        dw, dq = (saved[0], saved[1]) if ctx.has_w else (None, saved[0])
        gw = gL * dw if (dw is not None and ctx.needs_input_grad[0]) else None
        gq = (gL * dq).to(ctx.q_dtype) if ctx.needs_input_grad[1] else None
        return gw, gq, None, None, None, None
