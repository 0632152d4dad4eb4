"""GPU parity of the three-loop improved topological charge (Sec. IV.C) and
of the Wilson flow to given measurement times (Sec. IV.B) against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

from _helpers import flux_field

pytestmark = pytest.mark.gpu


def _thermal(orc, dims, beta, seed, n=3):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 1)
    return U


@pytest.mark.parametrize("dims", [[6, 6, 4, 4], [4, 4, 8, 6], [8, 8, 8, 8]])
def test_improved_charge_parity(gpu, orc, dims):
    U = _thermal(orc, dims, 6.0, 3)
    ref = orc.topo_charge_improved(U, dims)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    got = gpu.mgq_topo_charge_improved(lat)
    assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref))), (got, ref)
    # the 1 x 1 part is the clover charge of mgq_topo_charge
    assert abs(got[1] - gpu.mgq_topo_charge(lat)[1]) < 1e-12
    for prec, tol in [("f32", 2e-5), ("f32c12", 5e-5)]:
        l2 = gpu.Lattice(dims, prec)
        l2.from_numpy(U)
        g2 = gpu.mgq_topo_charge_improved(l2)
        assert np.max(np.abs(g2 - ref)) < tol * max(1.0, np.max(np.abs(ref))), (prec, g2, ref)


def test_improved_charge_constant_flux(gpu):
    dims = [8, 6, 10, 8]
    U, f, g = flux_field(dims, 2, -1)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    got = gpu.mgq_topo_charge_improved(lat)
    V = U.shape[0]
    want = [V * np.sin(m * m * f) * np.sin(m * m * g) / (2 * np.pi**2) for m in (1, 2, 3)]
    assert np.max(np.abs(got[1:] - want)) < 1e-10
    assert abs(got[0] - (1.5 * want[0] - 0.6 * want[1] / 16 + 0.1 * want[2] / 81)) < 1e-10


@pytest.mark.parametrize("charge,code", [("clover", 0), ("improved", 1)])
def test_flow_times_parity_fp64(gpu, orc, charge, code):
    dims = [6, 4, 4, 6]
    U = _thermal(orc, dims, 6.0, 4)
    tm = [0.0, 0.033, 0.05, 0.077, 0.1]
    W = U.copy()
    E_ref, Q_ref = orc.wilson_flow_times(W, dims, 0.1, 0.01, tm, charge=code)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    E, Q = gpu.mgq_wilson_flow_times(lat, 0.1, 0.01, tm, charge=charge)
    assert np.max(np.abs(E - E_ref)) < 1e-11 * max(1.0, np.max(np.abs(E_ref)))
    assert np.max(np.abs(Q - Q_ref)) < 1e-11
    assert np.max(np.abs(lat.to_numpy() - W)) < 1e-11


def test_flow_times_on_grid_equals_fixed_step_flow(gpu):
    dims = [8, 8, 8, 8]
    lat = gpu.Lattice(dims, "f32c12", seed=5)
    gpu.mgq_init_links(lat, 1)
    gpu.mgq_update_sweeps(lat, 6.0, 0, 5, 1, 2)
    ref = gpu.copy_lattice(lat)
    E1, Q1 = gpu.mgq_wilson_flow(ref, 0.02, 10, 5)
    E2, Q2 = gpu.mgq_wilson_flow_times(lat, 0.2, 0.02, [0.0, 0.1, 0.2])
    assert np.array_equal(E1, E2) and np.array_equal(Q1, Q2)
    assert np.array_equal(lat.links.cpu().numpy(), ref.links.cpu().numpy())


def test_flow_times_argument_checks(gpu):
    lat = gpu.Lattice([4, 4, 4, 4], "f64")
    gpu.mgq_init_links(lat, 0)
    for tm in ([0.2, 0.1], [0.3], [-0.1]):
        with pytest.raises(gpu.MgqError):
            gpu.mgq_wilson_flow_times(lat, 0.25, 0.01, tm)
