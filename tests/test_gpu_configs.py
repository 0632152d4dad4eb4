"""End-to-end pipelines of the benchmarked configurations on the GPU.

* Multiscale step (Sec. II-IV): coarse 8^4 at beta = 5.7 prolongated to 16^4
  (transfer + APE stages to 0.001 % relative change), 50 rethermalisation
  sweeps (1 HB + 4 OR) at beta = 6.0, Wilson flow to t = 1, clover Q.
* HMC on 24^4 at beta = 6.0: force against finite differences of the action
  at full size (FP64), and the FP32 12-real trajectory loop from a hot start.
"""
import numpy as np
import pytest
import torch

from paper_1510_04675_gb300.autograd import wilson_action

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def coarse_8(orc):
    U = orc.init_links([8, 8, 8, 8], 1, seed=101)
    orc.update_chain(U, [8, 8, 8, 8], 5.7, 101, 0, 0, 40, 1, 4)
    return U


def test_multiscale_prolongation_fp64_full_size(gpu, orc, coarse_8):
    """8^4 -> 16^4 with the paper's stopping rule: same iteration counts and
    links as the oracle; 2x2 loops from even sites equal coarse plaquettes."""
    Uc = coarse_8
    ref, it_ref, sd_ref = orc.prolongate(Uc, [8, 8, 8, 8], 0.05, 1e-5, 10000)
    c = gpu.Lattice([8, 8, 8, 8], "f64")
    c.from_numpy(Uc)
    f = gpu.Lattice([16, 16, 16, 16], "f64")
    iters, sd = gpu.mgq_prolongate(c, f, 0.05, 1e-5, 10000)
    assert iters == it_ref, (iters, it_ref)
    assert np.max(np.abs(np.array(sd) - sd_ref) / np.abs(sd_ref)) < 1e-9
    G = f.to_numpy()
    assert np.max(np.abs(G - ref)) < 1e-8
    c2 = gpu.Lattice([8, 8, 8, 8], "f64")
    gpu.mgq_restrict(f, c2)
    assert np.array_equal(c2.to_numpy(), Uc)       # R(Q(U)) = U exactly


def test_multiscale_step_fp32_pipeline(gpu, orc, coarse_8):
    """The FP32 12-real multiscale step: prolongation, 50 sweeps at beta = 6.0,
    flow to t = 1.  The fine ensemble must rethermalise (plaquette moves from
    the smooth prolongated value to the beta = 6.0 equilibrium, compared with
    an oracle chain from the same prolongated field) and E(t) must fall."""
    Uc = coarse_8
    c = gpu.Lattice([8, 8, 8, 8], "f32c12", seed=5)
    c.from_numpy(Uc)
    f = gpu.Lattice([16, 16, 16, 16], "f32c12", seed=5)
    iters, sd = gpu.mgq_prolongate(c, f, 0.05, 1e-5, 10000)
    p0 = gpu.mgq_plaquette(f)
    pl = gpu.mgq_update_sweeps(f, 6.0, 0, 50, 1, 4, plaq_out=True)
    # oracle chain from its own prolongation of the same coarse field (FP64)
    Uf, it_ref, _ = orc.prolongate(Uc, [8, 8, 8, 8], 0.05, 1e-5, 10000)
    assert abs(p0 - orc.plaquette(Uf, [16] * 4)) < 1e-5
    po = orc.update_chain(Uf, [16] * 4, 6.0, 5, 0, 0, 50, 1, 4)
    tail_g, tail_o = pl[30:], po[30:]
    assert abs(tail_g.mean() - tail_o.mean()) < 5 * np.hypot(tail_g.std(), tail_o.std()) / np.sqrt(5) + 3e-4
    assert tail_g.mean() < p0 - 0.05                # the smooth prolongated field has rethermalised
    w = gpu.copy_lattice(f)
    E, Q = gpu.mgq_wilson_flow(w, 0.01, 100, 10)
    assert np.all(np.diff(E[1:]) < 0) and E[-1] < E[0]
    assert np.isfinite(Q).all()


def test_hmc_force_finite_differences_24(gpu, orc):
    dims, beta, h = [24, 24, 24, 24], 6.0, 1e-4
    lat = gpu.Lattice(dims, "f64", seed=31)
    gpu.mgq_init_links(lat, 1)
    gpu.mgq_update_sweeps(lat, beta, 0, 3, 1, 1)
    omega = lat.new_alg_field().requires_grad_(True)
    (g,) = torch.autograd.grad(wilson_action(omega, lat, beta), omega)
    gen = torch.Generator(device="cuda").manual_seed(3)
    v = torch.randn(omega.shape, dtype=torch.float64, device="cuda", generator=gen)
    gpu.zero_alg_padding(lat, v)
    fd = (wilson_action(h * v, lat, beta) - wilson_action(-h * v, lat, beta)).item() / (2 * h)
    assert abs(fd - torch.dot(g, v).item()) < 1e-6 * abs(fd)


def test_hmc_24_hot_start_fp32(gpu):
    """24^4, beta = 6.0, tau = 1, 20 steps of 0.05, FP32 12-real links, FP64 H:
    24 warm-up trajectories without accept/reject (Sec. IV.E), then dH falls to
    O(1-10) as the field thermalises and the unitarity of the links holds."""
    lat = gpu.Lattice([24, 24, 24, 24], "f32c12", seed=77, with_mom=True)
    gpu.mgq_init_links(lat, 1)
    dHs = []
    for traj in range(30):
        dH, acc = gpu.mgq_hmc_trajectory(lat, 6.0, 1.0, 20, traj, 0 if traj < 24 else 1)
        dHs.append(dH)
        if traj < 24:
            assert acc == 1
    assert abs(dHs[-1]) < abs(dHs[0])
    assert gpu.mgq_check_unitarity(lat) < 5e-6
    p = gpu.mgq_plaquette(lat)
    assert 0.4 < p < 0.65
