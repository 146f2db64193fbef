"""Differentiable rollout: ``torch.autograd.Function`` over the C ABI.

Forward runs ``fl_step_rk_checkpointed`` on a copy of theta0: the rollout
(fused stage kernels) storing a checkpoint every ``checkpoint_every`` steps
in a workspace kept for backward.  Backward runs
``fl_step_rk_adjoint_from_checkpoints``: each segment is recomputed from its
checkpoint with its stage states stored, and the hand-written adjoint stage
kernels run in reverse.
The limiter derivative is taken on the branch the forward evaluation takes.
Only theta0 receives a gradient (the velocity is a fixed input).
"""
from __future__ import annotations

import torch

from . import (fl_adjoint_workspace_size, fl_step_rk_adjoint_from_checkpoints,
               fl_step_rk_checkpointed)


class LimitedRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta0, u_f, mesh, limiter, dt, nsteps, rk_order=3, checkpoint_every=20):
        theta = theta0.detach().clone().contiguous()
        nb = fl_adjoint_workspace_size(mesh.handle, theta.dtype, rk_order, nsteps,
                                       checkpoint_every)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device=theta.device)
        fl_step_rk_checkpointed(mesh.handle, limiter, theta.dtype, rk_order, dt, nsteps,
                                checkpoint_every, theta, u_f, ws, nb)
        ctx.save_for_backward(u_f.detach(), ws)
        ctx.cfg = (mesh, limiter, dt, nsteps, rk_order, checkpoint_every, nb)
        return theta

    @staticmethod
    def backward(ctx, grad_out):
        u_f, ws = ctx.saved_tensors
        mesh, limiter, dt, nsteps, rk_order, every, nb = ctx.cfg
        lam_T = grad_out.contiguous()
        lam_0 = torch.empty_like(lam_T)
        fl_step_rk_adjoint_from_checkpoints(mesh.handle, limiter, lam_T.dtype, rk_order, dt,
                                            nsteps, every, u_f, lam_T, lam_0, ws, nb)
        return lam_0, None, None, None, None, None, None, None


def rollout(theta0, u_f, mesh, limiter, dt, nsteps, rk_order=3, checkpoint_every=20):
    """theta_T as a differentiable function of theta0."""
    return LimitedRollout.apply(theta0, u_f, mesh, limiter, dt, nsteps, rk_order,
                                checkpoint_every)
