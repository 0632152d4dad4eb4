"""GPU m x n Wilson loops and rethermalisation diagnostics against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_loops_parity(gpu, orc):
    dims = [6, 4, 8, 4]
    U = orc.init_links(dims, 1, seed=4)
    orc.update_chain(U, dims, 5.8, 4, 0, 0, 3, 1, 1)
    for prec, tol in [("f64", 1e-13), ("f32c12", 2e-6)]:
        lat = gpu.Lattice(dims, prec)
        lat.from_numpy(U)
        for m, n in [(1, 1), (2, 2), (1, 3), (3, 2)]:
            assert abs(gpu.mgq_wilson_loop(lat, m, n) - orc.wilson_loop(U, dims, m, n)) < tol
        assert np.max(np.abs(gpu.mgq_partial_loops(lat) - orc.partial_loops(U, dims))) < 10 * tol


def test_prolongated_field_diagnostics(gpu, orc):
    """After prolongation W2x2_0 is the coarse plaquette (Sec. III); rethermalisation
    drives the five displaced loops together (Sec. IV.E)."""
    dc = [8, 8, 8, 8]
    Uc = orc.init_links(dc, 1, seed=9)
    orc.update_chain(Uc, dc, 5.7, 9, 0, 0, 20, 1, 4)
    c = gpu.Lattice(dc, "f64")
    c.from_numpy(Uc)
    f = gpu.Lattice([16] * 4, "f64", seed=3)
    gpu.mgq_prolongate(c, f, 0.05, 0.0, 30)
    d0 = gpu.mgq_partial_loops(f)
    assert abs(d0[3] - orc.plaquette(Uc, dc)) < 1e-13
    spread0 = np.ptp(d0[3:8])
    gpu.mgq_update_sweeps(f, 6.0, 0, 30, 1, 4)
    d1 = gpu.mgq_partial_loops(f)
    assert np.ptp(d1[3:8]) < 0.1 * spread0


def test_multilevel_refinement(gpu, orc):
    """Two refinement levels 4^4 -> 8^4 -> 16^4 (Sec. I: several levels of
    refinement): restricting twice gives back the coarsest field exactly, and
    the 2x2 loops from even sites of each level are the plaquettes of the level
    below."""
    d4 = [4, 4, 4, 4]
    U4 = orc.init_links(d4, 1, seed=12)
    orc.update_chain(U4, d4, 5.5, 12, 0, 0, 10, 1, 4)
    l4 = gpu.Lattice(d4, "f64")
    l4.from_numpy(U4)
    l8 = gpu.Lattice([8] * 4, "f64", seed=1)
    l16 = gpu.Lattice([16] * 4, "f64", seed=2)
    gpu.mgq_prolongate(l4, l8, 0.05, 1e-5, 2000)
    gpu.mgq_update_sweeps(l8, 5.8, 0, 5, 1, 4)          # rethermalise the middle level
    p8 = gpu.mgq_plaquette(l8)
    gpu.mgq_prolongate(l8, l16, 0.05, 1e-5, 2000)
    assert abs(gpu.mgq_partial_loops(l16)[3] - p8) < 1e-13
    back8 = gpu.Lattice([8] * 4, "f64")
    gpu.mgq_restrict(l16, back8)
    assert np.array_equal(back8.to_numpy(), l8.to_numpy())
