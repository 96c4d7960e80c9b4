"""torch.autograd wrappers around the fast product and its adjoint.

QmcMatmul:   B = Y·A, backward dA = Yᵀ·dB through the adjoint kernel (the
             transposed circulant applied with the conjugate spectrum).
ExpMeanLoss: l = mean_{n,k} exp((Y·A)_nk) (the log-normal application's
             exponential, Section 3.3), with the cotangent exp(B)/(rows·t)
             formed inside the adjoint's first pass.
"""

from __future__ import annotations

import torch

from .qmc import Plan


class QmcMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A: torch.Tensor, plan: Plan):
        ctx.plan = plan
        return plan.matmul(A.contiguous())

    @staticmethod
    def backward(ctx, dB: torch.Tensor):
        dA = ctx.plan.matmul_backward(dB.contiguous().float())
        return dA, None


class ExpMeanLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A: torch.Tensor, plan: Plan):
        B, _, esum = plan.matmul(A.contiguous(), exp_sum=True)
        ctx.plan = plan
        ctx.save_for_backward(B)
        return (esum / float(B.numel())).to(torch.float32).reshape(())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        (B,) = ctx.saved_tensors
        dA = ctx.plan.matmul_backward(B, g_mode=1)
        return dA * g.to(dA.dtype), None


def qmc_matmul(A: torch.Tensor, plan: Plan) -> torch.Tensor:
    return QmcMatmul.apply(A, plan)


def exp_mean_loss(A: torch.Tensor, plan: Plan) -> torch.Tensor:
    return ExpMeanLoss.apply(A, plan)
