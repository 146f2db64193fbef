"""Differentiable rollout: ``torch.autograd.Function`` over the C ABI.

Forward runs ``fl_step_rk`` (nsteps fused stages per RK stage) on a copy of
theta0; backward runs ``fl_step_rk_adjoint``: the rollout is checkpointed
every ``checkpoint_every`` steps, each segment is recomputed with its stage
states stored, and the hand-written adjoint stage kernels run in reverse.
The limiter derivative is taken on the branch the forward evaluation takes.
Only theta0 receives a gradient (the velocity is a fixed input).
"""
from __future__ import annotations

import torch

from . import (fl_adjoint_workspace_size, fl_step_rk, fl_step_rk_adjoint, fl_workspace_size)


class LimitedRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta0, u_f, mesh, limiter, dt, nsteps, rk_order=3, checkpoint_every=20):
        theta = theta0.detach().clone().contiguous()
        nb = fl_workspace_size(mesh.handle, theta.dtype, rk_order)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=theta.device)
        fl_step_rk(mesh.handle, limiter, theta.dtype, rk_order, dt, nsteps, theta, u_f, ws, nb)
        ctx.save_for_backward(theta0.detach(), u_f.detach())
        ctx.cfg = (mesh, limiter, dt, nsteps, rk_order, checkpoint_every)
        return theta

    @staticmethod
    def backward(ctx, grad_out):
        theta0, u_f = ctx.saved_tensors
        mesh, limiter, dt, nsteps, rk_order, every = ctx.cfg
        lam_T = grad_out.contiguous()
        lam_0 = torch.empty_like(theta0)
        nb = fl_adjoint_workspace_size(mesh.handle, theta0.dtype, rk_order, nsteps, every)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=theta0.device)
        fl_step_rk_adjoint(mesh.handle, limiter, theta0.dtype, rk_order, dt, nsteps, every,
                           theta0, u_f, lam_T, lam_0, ws, nb)
        return lam_0, None, None, None, None, None, None, None


def rollout(theta0, u_f, mesh, limiter, dt, nsteps, rk_order=3, checkpoint_every=20):
    """theta_T as a differentiable function of theta0."""
    return LimitedRollout.apply(theta0, u_f, mesh, limiter, dt, nsteps, rk_order,
                                checkpoint_every)
