"""GPU parity of the HMC gauge force, momenta, leapfrog and Metropolis step
(Sec. IV.D, App. A) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1510_04675_gb300.api import alg_to_numpy

pytestmark = pytest.mark.gpu


def _thermal(orc, dims, beta, seed, n=3):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 1)
    return U


@pytest.mark.parametrize("dims", [[8, 8, 8, 8], [6, 4, 2, 6]])
def test_force_parity_fp64(gpu, orc, dims):
    U = _thermal(orc, dims, 5.7, 3)
    ref = orc.force(U, dims, 5.7)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    F = lat.new_alg_field()
    gpu.mgq_hmc_force(lat, 5.7, F)
    got = alg_to_numpy(lat, F)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("prec,dims", [("f32", [8, 8, 8, 8]), ("f32c12", [24, 24, 24, 24]),
                                       ("f32c12", [6, 6, 6, 6]),    # 6^4: V/2 = 648, a partly filled 32-site band
                                       ("f32c12", [2, 4, 2, 6])])   # x + nu = x - nu in directions 0 and 2
def test_force_fp32(gpu, orc, prec, dims):
    U = orc.init_links(dims, 1, seed=4)
    lat = gpu.Lattice(dims, prec)
    lat.from_numpy(U)
    F = lat.new_alg_field()
    gpu.mgq_hmc_force(lat, 6.0, F)
    got = alg_to_numpy(lat, F)
    ref = orc.force(U, dims, 6.0)
    assert np.max(np.abs(got - ref)) < 2e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32c12", 2e-5)])
def test_momentum_step_parity(gpu, orc, prec, tol):
    """The leapfrog's fused P-step: P <- P + eps F(U) on lat.mom (Sec. IV.D)."""
    dims, beta, eps = [6, 4, 4, 8], 5.9, 0.037
    U = _thermal(orc, dims, beta, 5)
    rng = np.random.default_rng(6)
    P0 = rng.standard_normal((U.shape[0], 4, 8))
    lat = gpu.Lattice(dims, prec, with_mom=True)
    lat.from_numpy(U)
    from paper_1510_04675_gb300.api import alg_from_numpy

    lat.mom.view(lat.real_dtype()).copy_(alg_from_numpy(lat, P0))
    gpu.mgq_hmc_momentum_step(lat, beta, eps)
    ref = P0 + eps * orc.force(U, dims, beta)
    assert np.max(np.abs(lat.mom_numpy() - ref)) < tol * max(1.0, np.max(np.abs(ref)))


def test_trajectory_parity_fp64(gpu, orc):
    dims, beta = [4, 4, 4, 4], 5.7
    U = _thermal(orc, dims, beta, 5)
    lat = gpu.Lattice(dims, "f64", seed=9, lattice_id=1, with_mom=True)
    lat.from_numpy(U)
    for traj in range(6):
        P = np.zeros((U.shape[0], 4, 8))
        dH_ref, acc_ref = orc.hmc_trajectory(U, dims, beta, 1.0, 10, 9, 1, traj, 1, P)
        dH, acc = gpu.mgq_hmc_trajectory(lat, beta, 1.0, 10, traj, 1)
        assert acc == acc_ref, traj
        assert abs(dH - dH_ref) < 1e-9, (traj, dH, dH_ref)
        assert np.max(np.abs(lat.to_numpy() - U)) < 1e-11
        assert np.max(np.abs(lat.mom_numpy() - P)) < 1e-10


def test_warmup_and_rejection(gpu, orc):
    dims, beta = [4, 4, 2, 2], 5.7
    U = _thermal(orc, dims, beta, 6)
    lat = gpu.Lattice(dims, "f64", seed=2, with_mom=True)
    lat.from_numpy(U)
    dH, acc = gpu.mgq_hmc_trajectory(lat, beta, 4.0, 1, 0, 1)   # huge step: rejected, links restored
    assert dH > 50 and acc == 0
    assert np.array_equal(lat.to_numpy(), U)
    dH, acc = gpu.mgq_hmc_trajectory(lat, beta, 4.0, 1, 0, 0)   # warm-up: kept
    assert acc == 1 and not np.array_equal(lat.to_numpy(), U)


def test_trajectory_fp32_energy(gpu, orc):
    dims, beta = [8, 8, 8, 8], 6.0
    U = _thermal(orc, dims, beta, 7)
    P = np.zeros((U.shape[0], 4, 8))
    dH_ref, _ = orc.hmc_trajectory(U.copy(), dims, beta, 1.0, 20, 3, 0, 0, 0, P)
    lat = gpu.Lattice(dims, "f32", seed=3, with_mom=True)
    lat.from_numpy(U)
    dH, acc = gpu.mgq_hmc_trajectory(lat, beta, 1.0, 20, 0, 0)
    # FP32 links and momenta, FP64 Hamiltonian: dH agrees to the FP32 rounding of H ~ 1e5
    assert abs(dH - dH_ref) < 0.05, (dH, dH_ref)
    assert gpu.mgq_check_unitarity(lat) < 5e-6
