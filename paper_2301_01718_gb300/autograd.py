"""torch.autograd.Function over the HDM step of the library (the
differentiation form): the forward pass is hyrom_stage_full_step or
hyrom_stage_partial_step, the backward pass hyrom_stage_rk2_vjp.  Argument
marshalling only; the arithmetic runs in the library's kernels.

    step = HdmStep.apply(ctx, q_prev, k, s_hat)   # s_hat: cell bitmap or None
    loss = f(step); loss.backward()               # q_prev.grad = J^T dloss/dstep
"""
from __future__ import annotations

import torch

from . import hyrom


class HdmStep(torch.autograd.Function):
    """q_k = RK2_k(q_prev) on the cells of s_hat (every cell when s_hat is
    None) and q_prev on the others, for an FP64 Euler SSP-RK2 context."""

    @staticmethod
    def forward(fctx, ctx, q_prev, k, s_hat=None):
        q_prev = q_prev.detach().contiguous()
        if s_hat is None:
            out = torch.empty_like(q_prev)
            hyrom.hyrom_stage_full_step(ctx, q_prev, out, k)
        else:
            out = q_prev.clone()
            hyrom.hyrom_stage_partial_step(ctx, q_prev, out, s_hat, k)
        fctx.save_for_backward(q_prev)
        fctx.hy = (ctx, k, s_hat)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        (q_prev,) = fctx.saved_tensors
        ctx, k, s_hat = fctx.hy
        lam_out = grad_out.detach().contiguous()
        lam_in = torch.empty_like(q_prev)
        work = torch.empty(3 * q_prev.numel(), dtype=q_prev.dtype, device=q_prev.device)
        hyrom.hyrom_stage_rk2_vjp(ctx, q_prev, lam_out, lam_in, s_hat, k, work)
        return None, lam_in, None, None
