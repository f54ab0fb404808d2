"""torch.autograd wrapper of the lifted nnCANDELINC loss.

L = 1/2 ||X - I x_n F^(n) B^(n)||_F^2 (Eq. nnCANDELINC with the CPD of the
core substituted). The forward pass asks the library for the loss alone (one
pass over X); the backward pass calls the hand-written adjoint
(``candelinc_lifted_grad``), which recomputes the Tucker-compressed tensors
instead of saving them. X is data: it gets no gradient.
"""
from __future__ import annotations

import torch

from . import native


class LiftedLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, precision, *FB):
        d = X.dim()
        F, B = list(FB[:d]), list(FB[d:])
        loss, _, _ = native.candelinc_lifted_grad(X, F, B, precision=precision, grads=False)
        ctx.save_for_backward(X, *FB)
        ctx.precision = precision
        return torch.tensor(loss, dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, grad_out):
        X, *FB = ctx.saved_tensors
        d = X.dim()
        _, gF, gB = native.candelinc_lifted_grad(X, FB[:d], FB[d:], precision=ctx.precision)
        scale = grad_out.to(X.dtype)
        return (None, None, *[g * scale for g in gF], *[g * scale for g in gB])


def lifted_loss(X, F, B, precision=None):
    """Differentiable lifted loss: gradients flow to every F^(n) and B^(n)."""
    return LiftedLoss.apply(X, precision, *F, *B)
