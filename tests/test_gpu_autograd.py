"""torch.autograd.Function around the Wilson action whose backward is the
hand-written force kernel: checked against central finite differences of the
action (FP64, h = 1e-4) and against the oracle's force."""
import numpy as np
import pytest
import torch

from paper_1510_04675_gb300.api import alg_to_numpy
from paper_1510_04675_gb300.autograd import wilson_action

pytestmark = pytest.mark.gpu


def test_action_gradient_finite_differences(gpu, orc):
    dims, beta, h = [4, 4, 4, 6], 5.7, 1e-4
    U = orc.init_links(dims, 1, seed=12)
    orc.update_chain(U, dims, beta, 12, 0, 0, 3, 1, 1)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    omega = lat.new_alg_field().requires_grad_(True)
    S = wilson_action(omega, lat, beta)
    assert abs(S.item() - orc.action(U, dims, beta)) < 1e-9 * S.item()
    (g,) = torch.autograd.grad(S, omega)
    # the gradient is minus the oracle's force, link by link
    assert np.max(np.abs(alg_to_numpy(lat, g) + orc.force(U, dims, beta))) < 1e-11
    gen = torch.Generator(device="cuda").manual_seed(0)
    for _ in range(3):
        v = torch.randn(omega.shape, dtype=torch.float64, device="cuda", generator=gen)
        gpu.zero_alg_padding(lat, v)  # padding carries no links
        def cd(e):  # central difference, truncation error O(e^2)
            return (wilson_action(e * v, lat, beta) - wilson_action(-e * v, lat, beta)).item() / (2 * e)

        fd = (4 * cd(h / 2) - cd(h)) / 3  # Richardson: O(h^4)
        ad = torch.dot(g, v).item()
        assert abs(fd - ad) < 1e-7 * max(1.0, abs(ad)), (fd, ad)


def test_action_gradient_away_from_zero(gpu, orc):
    """At omega != 0 the backward is the true derivative d/domega S(exp(omega) U):
    it matches central differences (Richardson, h = 1e-4) for |omega| up to O(1)."""
    dims, beta, h = [4, 4, 2, 2], 6.0, 1e-4
    lat = gpu.Lattice(dims, "f64", seed=3)
    gpu.mgq_init_links(lat, 1)
    gen = torch.Generator(device="cuda").manual_seed(1)
    base = torch.randn(4 * 2 * 8 * lat.site_stride, dtype=torch.float64, device="cuda", generator=gen)
    gpu.zero_alg_padding(lat, base)
    v = torch.randn(base.shape, dtype=torch.float64, device="cuda", generator=gen)
    gpu.zero_alg_padding(lat, v)
    for scale in (1e-2, 0.3, 1.0):
        omega = (scale * base).requires_grad_(True)
        (g,) = torch.autograd.grad(wilson_action(omega, lat, beta), omega)
        w0 = omega.detach()

        def cd(e):
            return (wilson_action(w0 + e * v, lat, beta) - wilson_action(w0 - e * v, lat, beta)).item() / (2 * e)

        fd = (4 * cd(h / 2) - cd(h)) / 3
        ad = torch.dot(g, v).item()
        assert abs(fd - ad) < 1e-7 * max(1.0, abs(ad)), (scale, fd, ad)
