"""PyTorch autograd over the C ABI: the weighted bond force and its adjoint,
and the loss of a dynamic run with its micromodulus gradient.

``PDForce`` wraps ``pd_force`` (forward) and ``pd_force_adjoint`` (backward) of a
plan, so any torch computation built from force evaluations differentiates
through the library's kernels: the backward of L = F(u, s) is one fused
FFT-convolution pass that returns both (dL/du)^T gL and (dL/ds)^T gL.

``verlet_loss`` is the inverse-problem driver: ``pd_verlet_loss_grad`` runs the
velocity-Verlet dynamics (Eq. 83-84 with w = 0) under a spatially varying
micromodulus c(x) (bond factor s s' with s = sqrt(c), c relative to the plan's
micromodulus; with bond breaking when the plan has a critical energy), the
loss ||u(T) - u_target||^2, and, in the same call, the reverse sweep over
states recomputed from checkpoints every ``checkpoint_every`` steps. The
function here only marshals the tensors; every step runs in the library.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import pd as _pd


class PDForce(torch.autograd.Function):
    """L = pd_force(plan, u, s); backward = pd_force_adjoint."""

    @staticmethod
    def forward(ctx, u: torch.Tensor, s: Optional[torch.Tensor], plan: "_pd.Plan"):
        u = u.contiguous()
        s = None if s is None else s.contiguous()
        L = plan.force(u, s=s)
        ctx.plan = plan
        ctx.has_s = s is not None
        if s is None:
            ctx.save_for_backward(u)
        else:
            ctx.save_for_backward(u, s)
        return L

    @staticmethod
    def backward(ctx, gL: torch.Tensor):
        if ctx.has_s:
            u, s = ctx.saved_tensors
        else:
            (u,) = ctx.saved_tensors
            s = None
        want_gu = ctx.needs_input_grad[0]
        want_gs = ctx.has_s and ctx.needs_input_grad[1]
        if not (want_gu or want_gs):
            return None, None, None
        gu, gs = ctx.plan.force_adjoint(u, gL.contiguous(), s=s, want_gu=want_gu, want_gs=want_gs)
        return gu, gs, None


def pd_force(plan: "_pd.Plan", u: torch.Tensor, s: Optional[torch.Tensor] = None) -> torch.Tensor:
    return PDForce.apply(u, s, plan)


class VerletLoss(torch.autograd.Function):
    """J = pd_verlet_loss_grad(plan, c, ...); dJ/dc from the same call."""

    @staticmethod
    def forward(ctx, c: torch.Tensor, plan: "_pd.Plan", u_target: torch.Tensor, impulse: Optional[torch.Tensor],
                b: Optional[torch.Tensor], lam0: Optional[torch.Tensor], dt: float, nsteps: int,
                checkpoint_every: int):
        loss, grad = plan.verlet_loss_grad(c.contiguous(), u_target.contiguous(), dt, nsteps,
                                           checkpoint_every=checkpoint_every, lam0=lam0, b=b, b0=impulse,
                                           want_grad=ctx.needs_input_grad[0])
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=c.device))
        return torch.tensor(loss, dtype=c.dtype, device=c.device)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return grad * gJ, None, None, None, None, None, None, None, None


def verlet_loss(plan: "_pd.Plan", c: torch.Tensor, u_target: torch.Tensor, impulse: Optional[torch.Tensor],
                dt: float, nsteps: int, checkpoint_every: int = 10, b: Optional[torch.Tensor] = None,
                lam0: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Loss ||u(T) - u_target||^2 after nsteps of velocity Verlet from rest.

    ``impulse`` is a body force on the first step only, ``b`` a constant one;
    c is the micromodulus field relative to the plan's (bond factor
    sqrt(c c')); ``lam0`` an initial integrity index (bond breaking follows the
    plan's critical energy density)."""
    return VerletLoss.apply(c, plan, u_target, impulse, b, lam0, dt, nsteps, checkpoint_every)
