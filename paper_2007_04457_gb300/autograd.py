"""torch.autograd wrappers over the decomposition and recomposition.

Both maps are linear, so their backward passes are the transposed maps,
computed by the hand-written adjoint kernels (mgard_decompose_adjoint /
mgard_recompose_adjoint).  Nothing is saved for backward: each level of the
transpose is recomputed from the cotangent alone.
"""
from __future__ import annotations

import torch

from .mgard import Plan


class Decompose(torch.autograd.Function):
    """y = decompose(u); dL/du = decompose^T(dL/dy)."""

    @staticmethod
    def forward(ctx, u: torch.Tensor, plan: Plan):
        ctx.plan = plan
        out = u.detach().contiguous().clone()
        plan.decompose(out)
        return out

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        g = grad.contiguous().clone()
        ctx.plan.decompose_adjoint(g)
        return g, None


class Recompose(torch.autograd.Function):
    """u = recompose(y); dL/dy = recompose^T(dL/du)."""

    @staticmethod
    def forward(ctx, c: torch.Tensor, plan: Plan):
        ctx.plan = plan
        out = c.detach().contiguous().clone()
        plan.recompose(out)
        return out

    @staticmethod
    def backward(ctx, grad: torch.Tensor):
        g = grad.contiguous().clone()
        ctx.plan.recompose_adjoint(g)
        return g, None


def decompose(u: torch.Tensor, plan: Plan) -> torch.Tensor:
    return Decompose.apply(u, plan)


def recompose(c: torch.Tensor, plan: Plan) -> torch.Tensor:
    return Recompose.apply(c, plan)


def masked_reconstruction_loss(u: torch.Tensor, plan: Plan, mask: torch.Tensor) -> torch.Tensor:
    """||recompose(mask * decompose(u)) - u||^2: the error of reconstructing u
    from the coefficients the mask keeps."""
    r = recompose(mask * decompose(u, plan), plan) - u
    return (r * r).sum()
