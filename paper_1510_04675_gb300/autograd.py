"""torch.autograd wrappers whose backward passes are libmgq's hand-written
adjoint kernels.

WilsonAction: S(omega) = S_W(exp(omega) U) for an su(3) algebra field omega
(momentum layout, one 8-vector per link) around the lattice's current links.
The forward applies the exact exponential (mgq_link_exp_update) to a copy and
evaluates the Wilson action in FP64 (Sec. III); the backward is the gauge
force kernel (mgq_hmc_force): dS/domega_a = -F_a, the Lie derivative of S at
exp(omega) U.  That is the exact gradient at omega = 0 (and the
left-trivialised gradient elsewhere), which is what HMC and the gradient flow
use.
"""
from __future__ import annotations

import torch

from . import api


class WilsonAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, omega: torch.Tensor, lat: "api.Lattice", beta: float) -> torch.Tensor:
        moved = api.copy_lattice(lat)
        api.mgq_link_exp_update(moved, omega.detach().contiguous(), 1.0)
        plaq = api.mgq_plaquette(moved)
        ctx.moved, ctx.beta = moved, float(beta)
        S = float(beta) * 6.0 * moved.volume * (1.0 - plaq)
        return torch.tensor(S, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(ctx, grad_S: torch.Tensor):
        F = ctx.moved.new_alg_field()
        api.mgq_hmc_force(ctx.moved, ctx.beta, F)
        g = (-F.double() * grad_S).to(F.dtype)
        return g, None, None


def wilson_action(omega: torch.Tensor, lat: "api.Lattice", beta: float) -> torch.Tensor:
    return WilsonAction.apply(omega, lat, beta)
