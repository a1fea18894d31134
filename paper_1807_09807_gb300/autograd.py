"""torch.autograd wrappers of the TMOP kernels.

    F = tmop_energy(x, ctx)          # eq. (2.4), a 0-d float64 tensor on x's device
    F.backward()                      # x.grad = dF/dx by the adjoint gradient kernel

The backward of the energy is the library's gradient kernel (the gradient
formula of Section 3.4); the backward of the gradient is the matrix-free
Hessian action (the Hessian of Section 3.4 is symmetric), so double backward
and Hessian-vector products through torch also run on the CUDA kernels.

Fixed dofs are constants of the problem: their derivatives are returned as 0.
"""
from __future__ import annotations

import torch

from . import tmop as _tm


class TMOPGradient(torch.autograd.Function):
    """g = dF/dx (free dofs), with backward v -> H(x) v."""

    @staticmethod
    def forward(ctx, x, tctx):
        ctx.tctx = tctx
        ctx.save_for_backward(x)
        return tctx.gradient(x.contiguous())

    @staticmethod
    def backward(ctx, v):
        (x,) = ctx.saved_tensors
        return ctx.tctx.hess_apply(x.contiguous(), v.contiguous()), None


class TMOPEnergy(torch.autograd.Function):
    """F(x) as a 0-d tensor; backward grad_out * dF/dx."""

    @staticmethod
    def forward(ctx, x, tctx):
        ctx.tctx = tctx
        ctx.save_for_backward(x)
        F = torch.empty((), dtype=torch.float64, device=x.device)
        md = torch.empty((), dtype=torch.float64, device=x.device)
        tctx.energy_device(x.contiguous(), F, md)
        return F

    @staticmethod
    def backward(ctx, grad_out):
        (x,) = ctx.saved_tensors
        g = TMOPGradient.apply(x, ctx.tctx)
        return grad_out * g, None


def tmop_energy(x: torch.Tensor, tctx: "_tm.Context") -> torch.Tensor:
    """Differentiable TMOP objective of the positions x [dim, nnode] (float64, CUDA)."""
    return TMOPEnergy.apply(x, tctx)
