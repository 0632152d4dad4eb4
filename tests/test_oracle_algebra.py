"""Oracle pins: SU(3) algebra, exponential, reunitarisation and projection."""
import numpy as np

from _helpers import expm, gell_mann, random_hermitian_traceless, random_su3, unitarity_violation


def test_reunit_fixes_su3_and_lands_in_su3(orc):
    rng = np.random.default_rng(1)
    for _ in range(20):
        U = random_su3(rng)
        assert np.max(np.abs(orc.reunit(U) - U)) < 1e-14
        M = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        assert unitarity_violation(orc.reunit(M)) < 1e-14


def test_expm_matches_scipy(orc):
    rng = np.random.default_rng(2)
    for scale in [1e-6, 0.05, 0.3, 1.0, 3.0, 7.0]:
        X = scale * (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))
        ref = expm(X)
        assert np.max(np.abs(orc.expm(X) - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
    X = 1j * random_hermitian_traceless(rng, 2.0)
    E = orc.expm(X)
    assert unitarity_violation(E) < 1e-13
    assert np.max(np.abs(orc.expm(-X) @ E - np.eye(3))) < 1e-13


def test_generators_are_i_lambda_over_2(orc):
    lam = gell_mann()
    for a in range(8):
        e = np.zeros(8)
        e[a] = 1.0
        Xa = orc.alg_to_mat(e)
        assert np.max(np.abs(Xa - 0.5j * lam[a])) < 1e-15
    rng = np.random.default_rng(3)
    p = rng.standard_normal(8)
    M = orc.alg_to_mat(p)
    assert np.max(np.abs(M + M.conj().T)) < 1e-15 and abs(np.trace(M)) < 1e-15
    assert np.allclose(orc.mat_to_alg(M), p, atol=1e-14)
    # -Tr(P^2) = sum p^2 / 2 : the kinetic-energy normalisation
    assert abs(-np.trace(M @ M).real - 0.5 * np.sum(p * p)) < 1e-13


def test_projection_fixes_su3_and_positive_multiples(orc):
    rng = np.random.default_rng(4)
    for _ in range(10):
        U = random_su3(rng)
        assert np.max(np.abs(orc.su3_project(U) - U)) < 1e-14
        assert np.max(np.abs(orc.su3_project(3.7 * U) - U)) < 1e-14


def test_projection_converges_to_the_maximiser(orc):
    # For M = H U with H positive hermitian, U in SU(3) maximises Re Tr(W M^+).
    rng = np.random.default_rng(5)
    for _ in range(5):
        U = random_su3(rng)
        H = np.eye(3) + random_hermitian_traceless(rng, 0.15) + 0.05 * np.eye(3)
        assert np.all(np.linalg.eigvalsh(H) > 0)
        M = H @ U
        prev = -np.inf
        for n in [0, 1, 2, 4, 8]:
            W = orc.su3_project(M, n)
            assert unitarity_violation(W) < 1e-13
            val = np.trace(W @ M.conj().T).real
            assert val >= prev - 1e-13
            prev = val
        assert np.max(np.abs(orc.su3_project(M, 200) - U)) < 1e-10
        # within the eight-pass default, the objective is within 1e-8 of its maximum
        top = np.trace(U @ M.conj().T).real
        assert top - np.trace(orc.su3_project(M, 8) @ M.conj().T).real < 1e-8 * abs(top)
