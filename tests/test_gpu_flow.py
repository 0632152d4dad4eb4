"""GPU parity of the clover observables and the Wilson flow (Sec. IV.B-C)."""
import numpy as np
import pytest

from _helpers import flux_field

pytestmark = pytest.mark.gpu


def _thermal(orc, dims, beta, seed, n=3):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 1)
    return U


def test_clover_parity(gpu, orc):
    dims = [6, 6, 4, 4]
    U = _thermal(orc, dims, 6.0, 1)
    E_ref, Q_ref = orc.clover_EQ(U, dims)
    for prec, tol in [("f64", 1e-12), ("f32", 2e-6), ("f32c12", 5e-6)]:
        lat = gpu.Lattice(dims, prec)
        lat.from_numpy(U)
        E, Q = gpu.mgq_topo_charge(lat)
        assert abs(E - E_ref) < tol * max(1, abs(E_ref)) and abs(Q - Q_ref) < tol * 10, (prec, E, E_ref, Q, Q_ref)


def test_clover_constant_flux(gpu):
    dims = [4, 6, 4, 8]
    U, f, g = flux_field(dims, 1, 2)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    E, Q = gpu.mgq_topo_charge(lat)
    assert abs(E - 2 * (np.sin(f) ** 2 + np.sin(g) ** 2)) < 1e-12
    assert abs(Q - U.shape[0] * np.sin(f) * np.sin(g) / (2 * np.pi**2)) < 1e-11


def test_flow_parity_fp64(gpu, orc):
    dims = [6, 4, 4, 6]
    U = _thermal(orc, dims, 6.0, 2)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    E_ref, Q_ref = orc.wilson_flow(U, dims, 0.02, 10, 5)
    E, Q = gpu.mgq_wilson_flow(lat, 0.02, 10, 5)
    assert np.max(np.abs(E - E_ref)) < 1e-11 and np.max(np.abs(Q - Q_ref)) < 1e-11
    assert np.max(np.abs(lat.to_numpy() - U)) < 1e-11


def test_flow_fp32(gpu, orc):
    dims = [8, 8, 8, 8]
    U = _thermal(orc, dims, 6.0, 3)
    E_ref, Q_ref = orc.wilson_flow(U.copy(), dims, 0.01, 20, 10)
    for prec in ("f32", "f32c12"):
        lat = gpu.Lattice(dims, prec)
        lat.from_numpy(U)
        E, Q = gpu.mgq_wilson_flow(lat, 0.01, 20, 10)
        assert np.max(np.abs(E - E_ref) / E_ref) < 2e-5, (prec, E, E_ref)
        assert np.max(np.abs(Q - Q_ref)) < 1e-3
