"""torch.autograd wrapper of kura_adjoint: the terminal loss of an RK4 trajectory as a differentiable
function of (theta0, omega, K).

The forward call runs the library's checkpointed discrete adjoint (kura_adjoint), which returns the loss
together with all three gradients; backward scales the saved gradients by the incoming gradient.  All
arithmetic runs in libkura's kernels.
"""
from __future__ import annotations

import torch

from . import kura


class KuraRK4Loss(torch.autograd.Function):
    """loss = KuraRK4Loss.apply(theta0, omega, K, system, step, n_steps, ckpt_every, loss_kind, target)

    theta0, omega: float64 CUDA tensors of length n (user order); K: float64 0-d tensor.
    system: a kura.Kuramoto handle created with precision=kura.PREC_MIXED on the same graph.
    loss_kind 0: 1 - r(theta(T)); 1: 1/2 ||theta(T) - target||^2.
    The handle runs the adjoint with the given omega and K and gets its previous omega and K back afterwards.
    """

    @staticmethod
    def forward(ctx, theta0, omega, K, system, step, n_steps, ckpt_every=64, loss_kind=0, target=None):
        prev_omega, prev_K = system.omega, system.K
        system.set_param(omega=omega.detach().contiguous(), K=float(K))
        try:
            loss, g_om, g_K, g_th = system.adjoint(theta0.detach().contiguous(), step, n_steps, ckpt_every,
                                                   loss_kind,
                                                   None if target is None else target.detach().contiguous())
        finally:
            system.set_param(omega=prev_omega, K=prev_K)
        ctx.save_for_backward(g_th, g_om, torch.tensor(g_K, dtype=torch.float64, device=theta0.device))
        return torch.tensor(loss, dtype=torch.float64, device=theta0.device)

    @staticmethod
    def backward(ctx, grad_out):
        g_th, g_om, g_K = ctx.saved_tensors
        return grad_out * g_th, grad_out * g_om, grad_out * g_K, None, None, None, None, None, None
