"""``torch.autograd.Function`` around the library's loss and adjoint.

The forward pass calls ``sos_loss_grad`` once; the gradient 2 H(c - p) A that
it returns is saved and scaled by the incoming gradient in backward, so the
adjoint kernel runs exactly once per forward.
"""
from __future__ import annotations

import torch

from .engine import Plan


class SOSLossGrad(torch.autograd.Function):
    """loss(A) = 1/2 ||c(A) - p||^2 (Eq. 2 of the paper, scaled by 1/2)."""

    @staticmethod
    def forward(ctx, A: torch.Tensor, p: torch.Tensor, plan: Plan, prec: str = "fp32"):
        loss, _, grad = plan.loss_grad(A.detach().contiguous(), p, prec=prec,
                                       want_grad=A.requires_grad)
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=A.device))
        return loss.to(A.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        if grad.numel() == 0:
            return None, None, None, None
        return grad_out.to(grad.dtype) * grad, None, None, None


def sos_loss(A: torch.Tensor, p: torch.Tensor, plan: Plan, prec: str = "fp32") -> torch.Tensor:
    return SOSLossGrad.apply(A, p, plan, prec)
