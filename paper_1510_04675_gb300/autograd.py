"""torch.autograd wrappers whose backward passes are libmgq's hand-written
adjoint kernels.

WilsonAction: S(omega) = S_W(exp(omega) U) for an su(3) algebra field omega
(momentum layout, one 8-vector per link) around the lattice's current links.
The forward applies the exact exponential (mgq_link_exp_update) to a copy and
evaluates the Wilson action in FP64 (Sec. III); the backward is the gauge
force kernel (mgq_hmc_force), -F_a = the Lie derivative of S at exp(omega) U,
pulled back to omega through the adjoint differential of the exponential
(mgq_exp_vjp): dS/domega = J(omega)^T (-F).  At omega = 0, J is the identity
and the gradient is minus the HMC force.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


class WilsonAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, omega: torch.Tensor, lat: "api.Lattice", beta: float) -> torch.Tensor:
        moved = api.copy_lattice(lat)
        api.mgq_link_exp_update(moved, omega.detach().contiguous(), 1.0)
        plaq = api.mgq_plaquette(moved)
        ctx.moved, ctx.beta, ctx.omega = moved, float(beta), omega.detach().contiguous()
        S = float(beta) * 6.0 * moved.volume * (1.0 - plaq)
        return torch.tensor(S, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(ctx, grad_S: torch.Tensor):
        F = ctx.moved.new_alg_field()
        api.mgq_hmc_force(ctx.moved, ctx.beta, F)
        api.mgq_exp_vjp(ctx.moved, ctx.omega, F, F)
        g = (-F.double() * grad_S).to(F.dtype)
        return g, None, None


def wilson_action(omega: torch.Tensor, lat: "api.Lattice", beta: float) -> torch.Tensor:
    return WilsonAction.apply(omega, lat, beta)


_NO_TIMES = np.zeros(0)


def _flow_steps(lat, eps, n):
    """n fixed flow steps of size eps with no measurement (mgq_wilson_flow_times
    with one step per call and no measurement times: nothing is read back, so
    the host does not wait)."""
    for _ in range(n):
        api.mgq_wilson_flow_times(lat, eps, eps, _NO_TIMES)


class FlowedObservable(torch.autograd.Function):
    """L(omega) = O(W_t), W_t the Wilson flow (n_steps fixed steps of size eps,
    Sec. IV.B) of exp(omega) U, O one of
      "S": the Wilson action at coupling beta,
      "E": the clover energy density, "Q": the clover topological charge.

    The cotangent at the unflowed field exp(omega) U is pulled back to omega
    by mgq_exp_vjp, so the gradient is the true omega-derivative.

    Forward: the flow kernels, keeping a copy of the field every
    `checkpoint_every` steps (default sqrt(n_steps)).  Backward: the gradient
    of O at W_t -- the force kernel for S, mgq_clover_vjp for E and Q -- is
    pulled back step by step with the adjoint-flow kernels
    (mgq_wilson_flow_step_adjoint); each segment between checkpoints is
    recomputed forward to recover the start of every step.  Memory: the
    checkpoints plus one segment of link fields.
    """

    @staticmethod
    def forward(ctx, omega, lat, observable, eps, n_steps, beta=6.0, checkpoint_every=None):
        import math

        k = int(checkpoint_every or max(1, int(math.isqrt(max(1, n_steps)))))
        W = api.copy_lattice(lat)
        api.mgq_link_exp_update(W, omega.detach().contiguous(), 1.0)
        ckpts = []
        done = 0
        while done < n_steps:
            ckpts.append((done, W.links.clone()))
            m = min(k, n_steps - done)
            _flow_steps(W, eps, m)
            done += m
        if observable == "S":
            value = float(beta) * 6.0 * W.volume * (1.0 - api.mgq_plaquette(W))
        else:
            E, Q = api.mgq_topo_charge(W)
            value = E if observable == "E" else Q
        ctx.W, ctx.ckpts, ctx.k, ctx.omega = W, ckpts, k, omega.detach().contiguous()
        ctx.obs, ctx.beta, ctx.eps, ctx.n = observable, float(beta), float(eps), int(n_steps)
        return torch.tensor(value, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(ctx, grad_L):
        W = ctx.W
        lam = W.new_alg_field()
        if ctx.obs == "S":
            api.mgq_hmc_force(W, ctx.beta, lam)      # F = -dS/domega at W_t
            lam.mul_(-1.0)
        else:
            api.mgq_clover_vjp(W, ctx.obs, 1.0, lam)
        scratch = api.flow_adjoint_scratch(W)
        seg = api.copy_lattice(W)
        for start, links in reversed(ctx.ckpts):
            m = min(ctx.n - start, ctx.k)
            seg.links.copy_(links)
            starts = []
            for _ in range(m):
                starts.append(seg.links.clone())
                _flow_steps(seg, ctx.eps, 1)
            for w0 in reversed(starts):
                seg.links.copy_(w0)
                api.mgq_wilson_flow_step_adjoint(seg, ctx.eps, lam, scratch)
        api.mgq_exp_vjp(W, ctx.omega, lam, lam)   # from exp(omega) U back to omega
        return (lam.double() * grad_L).to(lam.dtype), None, None, None, None, None, None


def flowed_observable(omega, lat, observable, eps, n_steps, beta=6.0, checkpoint_every=None):
    """Differentiable O(W_t) for O in {"S", "E", "Q"} (see FlowedObservable)."""
    return FlowedObservable.apply(omega, lat, observable, eps, n_steps, beta, checkpoint_every)


def flowed_wilson_action(omega, lat, beta, eps, n_steps, checkpoint_every=None):
    return FlowedObservable.apply(omega, lat, "S", eps, n_steps, beta, checkpoint_every)
