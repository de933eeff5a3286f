"""torch.autograd wrapper of qtt_grad: the mean final product J as a
differentiable function of the model parameters.

    theta = torch.tensor([omega, da, gamma, a_0, ..., b_0, ...], dtype=torch.float64, requires_grad=True)
    J = MeanProduct.apply(theta, params, nsteps, ckpt_every)
    J.backward()          # theta.grad = dJ/dtheta from the discrete adjoint

theta follows grad_param_names(params): Omega, Da, gamma, the velocity
mode amplitudes, the initial-condition mode amplitudes.  The forward call
runs the whole adjoint (one qtt_grad call: forward sweep with checkpoints,
backward sweep), so backward only scales the stored gradient.  The time
step params['dt'] is held fixed.  Only argument marshalling happens here.
"""
from __future__ import annotations

import copy

import torch

from ._binding import Context, grad_param_names


def params_with_theta(params: dict, theta) -> dict:
    """A copy of params with the values of theta in the grad_param_names order."""
    names = grad_param_names(params)
    vals = [float(v) for v in theta]
    if len(vals) != len(names):
        raise ValueError(f"theta has {len(vals)} entries, expected {len(names)} ({names})")
    p = copy.deepcopy(params)
    for n, v in zip(names, vals):
        if n.startswith("umode"):
            p["umodes"][int(n[5:])]["amp"] = v
        elif n.startswith("icmode"):
            p["icmodes"][int(n[6:])]["amp"] = v
        else:
            p[n] = v
    return p


class MeanProduct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, params, nsteps, ckpt_every=0):
        p = params_with_theta(params, theta.detach().cpu().tolist())
        with Context(p) as c:
            J, g = c.grad(int(nsteps), int(ckpt_every))
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None
