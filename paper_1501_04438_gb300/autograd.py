"""Differentiable forms of the apply (PyTorch autograd, hand-written backward).

The discrete operator of a plan is u = C F^-1 diag(m) F P rho, with P the zero
padding, C the crop (its adjoint) and m a real multiplier even in k, so it is
symmetric: the backward of u = apply(rho) is grad_rho = apply(grad_u).

hartree_energy(psi, plan) = 1/2 h^d sum |psi|^2 (U |psi|^2); its gradient with
respect to psi is 2 h^d u psi in PyTorch's convention for a real loss
(dE/dRe psi + i dE/dIm psi).  Both energy and gradient come from one library
call (gsm_hartree); the backward scales the stored gradient.
"""
from __future__ import annotations

import torch


class GSMApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, plan):
        ctx.plan = plan
        return plan.apply(rho.contiguous())

    @staticmethod
    def backward(ctx, grad_u):
        return ctx.plan.apply(grad_u.contiguous()), None


class _Hartree(torch.autograd.Function):
    @staticmethod
    def forward(ctx, psi, plan):
        energy, u, grad = plan.hartree(psi.contiguous())
        ctx.save_for_backward(grad)
        return energy

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None


def hartree_energy(psi, plan):
    """E = 1/2 h^d <|psi|^2, U * |psi|^2> (differentiable in psi)."""
    return _Hartree.apply(psi, plan)
