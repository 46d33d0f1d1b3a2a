"""PyTorch autograd over the C ABI: the weighted bond force and its adjoint.

``PDForce`` wraps ``pd_force`` (forward) and ``pd_force_adjoint`` (backward) of a
plan, so any torch computation built from force evaluations differentiates
through the library's kernels: the backward of L = F(u, s) is one fused
FFT-convolution pass that returns both (dL/du)^T gL and (dL/ds)^T gL.

``verlet_loss`` is the inverse-problem driver: velocity-Verlet dynamics
(Eq. 67; with chi_Omega = chi_B and w = 0 the EC update of Eq. 83-84 reduces to
it) under a spatially varying micromodulus c(x) = c0 s(x)^2 (bond factor
s s' = sqrt(c c')/c0), and a loss on the final displacement. Gradients with
respect to c go through ``PDForce``; activations are recomputed per segment of
``checkpoint_every`` steps (torch.utils.checkpoint), so memory holds one
(u, v) pair per segment instead of one per step.
"""
from __future__ import annotations

from typing import Optional

import torch
from torch.utils.checkpoint import checkpoint

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


def verlet_loss(plan: "_pd.Plan", c: torch.Tensor, u_target: torch.Tensor, impulse: torch.Tensor, dt: float,
                nsteps: int, rho: float = 1.0, c0: float = 1.0, checkpoint_every: int = 10) -> torch.Tensor:
    """Loss ||u(T) - u_target||^2 after nsteps of velocity Verlet from rest.

    The body force is ``impulse`` on the first step and zero afterwards. The
    micromodulus field enters as the node weight s = sqrt(c / c0).
    """
    s = torch.sqrt(c / c0)
    u = torch.zeros_like(u_target)
    v = torch.zeros_like(u_target)
    h = dt / (2.0 * rho)

    def segment(u, v, s, k0, k1):
        a = pd_force(plan, u, s)
        if k0 == 0:
            a = a + impulse
        for k in range(k0, k1):
            v = v + h * a
            u = u + dt * v
            a = pd_force(plan, u, s)
            v = v + h * a
        return u, v

    k = 0
    while k < nsteps:
        k1 = min(nsteps, k + checkpoint_every)
        if checkpoint_every > 0 and torch.is_grad_enabled():
            u, v = checkpoint(segment, u, v, s, k, k1, use_reentrant=False)
        else:
            u, v = segment(u, v, s, k, k1)
        k = k1
    return ((u - u_target) ** 2).sum()
