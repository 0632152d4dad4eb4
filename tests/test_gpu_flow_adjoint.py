"""Adjoint Wilson flow: the vector-Jacobian product of the flow generator, one
reverse RK3 step, and the checkpointed multi-step autograd.Function, all
against central finite differences of forward quantities (FP64)."""
import numpy as np
import pytest
import torch

from paper_1510_04675_gb300 import api
from paper_1510_04675_gb300.autograd import flowed_wilson_action

pytestmark = pytest.mark.gpu


def _field(gpu, dims, seed, sweeps=2):
    lat = gpu.Lattice(dims, "f64", seed=seed)
    gpu.mgq_init_links(lat, 1)
    gpu.mgq_update_sweeps(lat, 6.0, 0, sweeps, 1, 1)
    return lat


def _rand_alg(lat, gen, scale=1.0):
    v = torch.randn(4 * 2 * 8 * lat.site_stride, dtype=torch.float64, device="cuda", generator=gen) * scale
    api.zero_alg_padding(lat, v)
    return v


def _Z(gpu, lat):
    F = lat.new_alg_field()
    gpu.mgq_hmc_force(lat, 6.0, F)   # -(6/6) TA(W A) = Z(W)
    return F


def _moved(gpu, lat, v, h):
    m = gpu.copy_lattice(lat)
    gpu.mgq_link_exp_update(m, v, h)
    return m


def test_generator_vjp_matches_finite_differences(gpu):
    lat = _field(gpu, [4, 4, 2, 4], 3)
    gen = torch.Generator(device="cuda").manual_seed(5)
    psi, v = _rand_alg(lat, gen), _rand_alg(lat, gen)
    lam = lat.new_alg_field()
    gpu.mgq_flow_vjp(lat, psi, 1.0, lam)
    h = 1e-5
    def cd(e):  # central difference, truncation error O(e^2)
        return torch.dot(psi, (_Z(gpu, _moved(gpu, lat, v, e)) - _Z(gpu, _moved(gpu, lat, v, -e))) / (2 * e)).item()

    fd = (4 * cd(h / 2) - cd(h)) / 3  # Richardson: O(h^4)
    ad = torch.dot(lam, v).item()
    assert abs(fd - ad) < 1e-7 * max(1.0, abs(fd)), (fd, ad)


def _action(gpu, lat, beta=6.0):
    return beta * 6 * lat.volume * (1 - gpu.mgq_plaquette(lat))


def test_one_step_adjoint(gpu):
    lat = _field(gpu, [4, 4, 4, 2], 7)
    eps = 0.05
    W = gpu.copy_lattice(lat)
    gpu.mgq_wilson_flow(W, eps, 1, 2)
    lam = W.new_alg_field()
    gpu.mgq_hmc_force(W, 6.0, lam)
    lam.mul_(-1.0)                                   # dS/domega at W_eps
    scratch = gpu.flow_adjoint_scratch(lat)
    gpu.mgq_wilson_flow_step_adjoint(lat, eps, lam, scratch)
    gen = torch.Generator(device="cuda").manual_seed(9)
    v = _rand_alg(lat, gen)
    h = 1e-5

    def L(sign):
        m = _moved(gpu, lat, v, sign * h)
        gpu.mgq_wilson_flow(m, eps, 1, 2)
        return _action(gpu, m)

    fd = (L(1) - L(-1)) / (2 * h)
    ad = torch.dot(lam, v).item()
    assert abs(fd - ad) < 1e-6 * max(1.0, abs(fd)), (fd, ad)


@pytest.mark.parametrize("n_steps,every", [(10, 3), (6, 6)])
def test_checkpointed_flow_gradient(gpu, n_steps, every):
    lat = _field(gpu, [4, 4, 4, 4], 11)
    eps, beta = 0.02, 6.0
    omega = lat.new_alg_field().requires_grad_(True)
    L0 = flowed_wilson_action(omega, lat, beta, eps, n_steps, every)
    (g,) = torch.autograd.grad(L0, omega)
    gen = torch.Generator(device="cuda").manual_seed(13)
    v = _rand_alg(lat, gen)
    h = 1e-5
    fd = (flowed_wilson_action(h * v, lat, beta, eps, n_steps).item()
          - flowed_wilson_action(-h * v, lat, beta, eps, n_steps).item()) / (2 * h)
    ad = torch.dot(g, v).item()
    assert abs(fd - ad) < 1e-6 * max(1.0, abs(fd)), (fd, ad)


@pytest.mark.parametrize("obs", ["E", "Q"])
def test_clover_gradient(gpu, obs):
    lat = _field(gpu, [4, 4, 4, 4], 21, sweeps=3)
    lam = lat.new_alg_field()
    gpu.mgq_clover_vjp(lat, obs, 1.0, lam)
    gen = torch.Generator(device="cuda").manual_seed(22)
    v = _rand_alg(lat, gen)
    h = 1e-5
    idx = 0 if obs == "E" else 1
    fd = (gpu.mgq_topo_charge(_moved(gpu, lat, v, h))[idx] - gpu.mgq_topo_charge(_moved(gpu, lat, v, -h))[idx]) / (2 * h)
    ad = torch.dot(lam, v).item()
    assert abs(fd - ad) < 1e-6 * max(1e-3, abs(fd)), (fd, ad)


@pytest.mark.parametrize("obs", ["E", "Q"])
def test_flowed_clover_gradient(gpu, obs):
    from paper_1510_04675_gb300.autograd import flowed_observable

    lat = _field(gpu, [4, 4, 4, 4], 31, sweeps=3)
    eps, n = 0.02, 8
    omega = lat.new_alg_field().requires_grad_(True)
    (g,) = torch.autograd.grad(flowed_observable(omega, lat, obs, eps, n, checkpoint_every=3), omega)
    gen = torch.Generator(device="cuda").manual_seed(32)
    v = _rand_alg(lat, gen)
    h = 1e-5
    fd = (flowed_observable(h * v, lat, obs, eps, n).item() - flowed_observable(-h * v, lat, obs, eps, n).item()) / (2 * h)
    ad = torch.dot(g, v).item()
    assert abs(fd - ad) < 1e-6 * max(1e-3, abs(fd)), (fd, ad)


@pytest.mark.parametrize("obs", ["S", "Q"])
def test_flowed_gradient_away_from_zero(gpu, obs):
    """At omega != 0 the backward is the true derivative of O(flow(exp(omega) U))."""
    from paper_1510_04675_gb300.autograd import flowed_observable

    lat = _field(gpu, [4, 4, 4, 4], 41, sweeps=3)
    eps, n = 0.02, 6
    gen = torch.Generator(device="cuda").manual_seed(42)
    w0 = _rand_alg(lat, gen, 0.5)
    omega = w0.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(flowed_observable(omega, lat, obs, eps, n, checkpoint_every=2), omega)
    v = _rand_alg(lat, gen)
    h = 1e-5
    fd = (flowed_observable(w0 + h * v, lat, obs, eps, n).item()
          - flowed_observable(w0 - h * v, lat, obs, eps, n).item()) / (2 * h)
    ad = torch.dot(g, v).item()
    assert abs(fd - ad) < 1e-6 * max(1e-3, abs(fd)), (fd, ad)
