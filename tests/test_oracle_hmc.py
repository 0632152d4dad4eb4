"""Oracle pins: HMC force against finite differences of the Wilson action,
momentum distribution, leapfrog reversibility, dH ~ eps^2 and the Creutz
equality <exp(-dH)> = 1 (Sec. IV.D, PQP leapfrog)."""
import numpy as np
import scipy.stats

from _helpers import expm, unitarity_violation

D4 = [4, 4, 4, 4]


def _thermal(orc, dims, beta, seed, n=4):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 1)
    return U


def test_force_is_minus_gradient_of_action(orc):
    beta, h = 5.7, 1e-4
    U = _thermal(orc, D4, beta, 21)
    F = orc.force(U, D4, beta)
    rng = np.random.default_rng(0)
    for _ in range(4):
        s, mu = int(rng.integers(U.shape[0])), int(rng.integers(4))
        for a in range(8):
            e = np.zeros(8)
            e[a] = 1.0
            Xa = orc.alg_to_mat(e)
            Up, Um = U.copy(), U.copy()
            Up[s, mu] = expm(h * Xa) @ U[s, mu]
            Um[s, mu] = expm(-h * Xa) @ U[s, mu]
            fd = -(orc.action(Up, D4, beta) - orc.action(Um, D4, beta)) / (2 * h)
            assert abs(fd - F[s, mu, a]) < 1e-6 * max(1.0, abs(F[s, mu, a]))


def test_momenta_are_standard_normal(orc):
    P = orc.mom_refresh(D4, 3, 1, 7)
    x = P.ravel()
    assert scipy.stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(orc.kinetic(P, D4) - 0.5 * np.sum(x * x)) < 1e-9


def test_leapfrog_reversibility(orc):
    beta = 5.7
    U0 = _thermal(orc, D4, beta, 22)
    P0 = orc.mom_refresh(D4, 22, 0, 1)
    U, P = U0.copy(), P0.copy()
    orc.leapfrog(U, P, D4, beta, 1.0, 10)
    assert np.max(np.abs(U - U0)) > 0.1
    P = -P
    orc.leapfrog(U, P, D4, beta, 1.0, 10)
    assert np.max(np.abs(U - U0)) < 1e-10
    assert np.max(np.abs(-P - P0)) < 1e-10
    assert unitarity_violation(U) < 1e-13


def test_energy_violation_scales_as_eps_squared(orc):
    beta = 5.7
    ratios = []
    for seed in (31, 32, 33):
        U0 = _thermal(orc, D4, beta, seed, 6)
        P0 = orc.mom_refresh(D4, seed, 0, 0)
        H0 = orc.kinetic(P0, D4) + orc.action(U0, D4, beta)
        dH = []
        for n in (8, 16, 32):
            U, P = U0.copy(), P0.copy()
            orc.leapfrog(U, P, D4, beta, 0.5, n)
            dH.append(orc.kinetic(P, D4) + orc.action(U, D4, beta) - H0)
        ratios += [dH[0] / dH[1], dH[1] / dH[2]]
    assert all(3.0 < r < 5.0 for r in ratios), ratios


def test_creutz_equality(orc):
    beta, dims = 5.7, [4, 4, 4, 4]
    U = _thermal(orc, dims, beta, 40, 10)
    vals, accs = [], []
    for traj in range(120):
        dH, acc = orc.hmc_trajectory(U, dims, beta, 1.0, 12, 40, 0, traj, 1)
        vals.append(np.exp(-dH))
        accs.append(acc)
    v = np.array(vals[10:])
    assert abs(v.mean() - 1) < 4 * v.std() / np.sqrt(v.size) + 1e-3
    assert 0.3 < np.mean(accs) <= 1.0


def test_rejection_restores_links(orc):
    beta = 5.7
    U0 = _thermal(orc, D4, beta, 50)
    # one very coarse step: |dH| is huge, so the Metropolis test rejects
    U = U0.copy()
    dH, acc = orc.hmc_trajectory(U, D4, beta, 4.0, 1, 50, 0, 0, 1)
    assert dH > 50 and acc == 0 and np.array_equal(U, U0)
    # warm-up mode (no accept/reject) keeps the proposal
    U = U0.copy()
    dH, acc = orc.hmc_trajectory(U, D4, beta, 4.0, 1, 50, 0, 0, 0)
    assert acc == 1 and not np.array_equal(U, U0)
