"""GPU parity of restriction, transfer and APE interpolation (Sec. III)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _coarse(orc, dims, beta=5.7, seed=1, n=4):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 2)
    return U


def test_transfer_and_restriction_exact(gpu, orc):
    dc = [4, 2, 4, 4]
    df = [2 * v for v in dc]
    Uc = _coarse(orc, dc)
    c = gpu.Lattice(dc, "f64")
    c.from_numpy(Uc)
    f = gpu.Lattice(df, "f64")
    iters, _ = gpu.mgq_prolongate(c, f, 0.05, 0.0, 0)  # transfer only
    assert iters == [0, 0, 0]
    assert np.array_equal(f.to_numpy(), orc.transfer(Uc, dc))
    c2 = gpu.Lattice(dc, "f64")
    gpu.mgq_restrict(f, c2)
    assert np.array_equal(c2.to_numpy(), Uc)


def test_prolongation_fixed_iterations_fp64(gpu, orc):
    dc = [2, 4, 2, 4]
    Uc = _coarse(orc, dc, seed=2)
    ref, it_ref, sd_ref = orc.prolongate(Uc, dc, 0.05, 0.0, 6)
    c = gpu.Lattice(dc, "f64")
    c.from_numpy(Uc)
    f = gpu.Lattice([2 * v for v in dc], "f64")
    iters, sd = gpu.mgq_prolongate(c, f, 0.05, 0.0, 6)
    assert iters == it_ref == [6, 6, 6]
    assert np.max(np.abs(f.to_numpy() - ref)) < 1e-11
    assert np.max(np.abs(np.array(sd) - sd_ref)) < 1e-10


def test_prolongation_stopping_rule_fp64(gpu, orc):
    dc = [4, 4, 2, 2]
    Uc = _coarse(orc, dc, seed=3)
    ref, it_ref, sd_ref = orc.prolongate(Uc, dc, 0.05, 1e-5, 5000)
    c = gpu.Lattice(dc, "f64")
    c.from_numpy(Uc)
    f = gpu.Lattice([2 * v for v in dc], "f64")
    iters, sd = gpu.mgq_prolongate(c, f, 0.05, 1e-5, 5000)
    assert iters == it_ref
    assert np.max(np.abs(np.array(sd) - sd_ref)) < 1e-9 * max(1, max(abs(v) for v in sd_ref))
    assert np.max(np.abs(f.to_numpy() - ref)) < 1e-9


@pytest.mark.parametrize("prec", ["f32", "f32c12"])
def test_prolongation_fp32(gpu, orc, prec):
    dc = [8, 8, 8, 8]   # the multiscale-step coarse lattice, prolongated to 16^4
    Uc = _coarse(orc, dc, seed=4, n=3)
    ref, it_ref, sd_ref = orc.prolongate(Uc, dc, 0.05, 0.0, 20)
    c = gpu.Lattice(dc, prec)
    c.from_numpy(Uc)
    f = gpu.Lattice([16, 16, 16, 16], prec)
    iters, sd = gpu.mgq_prolongate(c, f, 0.05, 0.0, 20)
    assert np.max(np.abs(np.array(sd) - sd_ref) / np.abs(sd_ref)) < 1e-4
    assert abs(gpu.mgq_plaquette(f) - orc.plaquette(ref, [16] * 4)) < 2e-6
