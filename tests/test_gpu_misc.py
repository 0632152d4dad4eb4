"""Checkpoint/resume, the Q-step entry point, and the non-unitary link check."""
import numpy as np
import pytest
import torch

from paper_1510_04675_gb300 import MgqError

pytestmark = pytest.mark.gpu


def test_checkpoint_resume_is_bit_exact(gpu, tmp_path):
    dims, beta = [6, 4, 4, 6], 5.9
    a = gpu.Lattice(dims, "f32c12", seed=5, lattice_id=2)
    gpu.mgq_init_links(a, 1)
    gpu.mgq_update_sweeps(a, beta, 0, 10, 1, 2)
    b = gpu.Lattice(dims, "f32c12", seed=5, lattice_id=2)
    gpu.mgq_init_links(b, 1)
    gpu.mgq_update_sweeps(b, beta, 0, 4, 1, 2)
    path = str(tmp_path / "cfg.mgq")
    gpu.save_checkpoint(b, path, beta, 4)
    del b
    c, beta_c, sweep = gpu.load_checkpoint(path)
    assert (beta_c, sweep) == (beta, 4)
    gpu.mgq_update_sweeps(c, beta_c, sweep, 6, 1, 2)
    assert torch.equal(a.links, c.links)
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0xFF
    open(path, "wb").write(raw)
    with pytest.raises(ValueError):
        gpu.load_checkpoint(path)


def test_link_exp_update_matches_oracle(gpu, orc):
    dims = [4, 4, 4, 4]
    U = orc.init_links(dims, 1, seed=8)
    P = orc.mom_refresh(dims, 8, 0, 3)
    lat = gpu.Lattice(dims, "f64", seed=8, with_mom=True)
    lat.from_numpy(U)
    # momenta through a trajectory-free route: build the algebra buffer from the oracle's numbers
    A = gpu.alg_from_numpy(lat, P)
    gpu.mgq_link_exp_update(lat, A, 0.3)
    orc.update_links(U, P, dims, 0.3)
    assert np.max(np.abs(lat.to_numpy() - U)) < 1e-13


def test_non_unitary_link_is_detected(gpu, orc):
    dims = [4, 4, 2, 2]
    U = orc.init_links(dims, 1, seed=2)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    assert gpu.mgq_check_unitarity(lat, 1e-10) < 1e-13
    U[7, 2] *= 1.001   # corrupted on the host
    lat.from_numpy(U)
    with pytest.raises(MgqError) as e:
        gpu.mgq_check_unitarity(lat, 1e-10)
    assert e.value.status == 6


def test_reunitarize_pass(gpu, orc):
    """Gram-Schmidt projection of every link (the reunitarisation of the update
    kernels): FP64 against the oracle's, FP32 with an FP32 or FP64 projection."""
    dims = [4, 4, 2, 6]
    rng = np.random.default_rng(9)
    U = orc.init_links(dims, 1, seed=9)
    M = U + 0.01 * (rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape))
    ref = np.stack([[orc.reunit(M[s, mu]) for mu in range(4)] for s in range(M.shape[0])])
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(M)
    gpu.mgq_reunitarize(lat)
    assert np.max(np.abs(lat.to_numpy() - ref)) < 1e-14
    for prec in ("f32", "f32c12"):
        for f64 in (False, True):
            l2 = gpu.Lattice(dims, prec)
            l2.from_numpy(M)
            gpu.mgq_reunitarize(l2, fp64_projection=f64)
            assert np.max(np.abs(l2.to_numpy() - ref)) < 2e-6, (prec, f64)
            assert gpu.mgq_check_unitarity(l2) < 1e-6
