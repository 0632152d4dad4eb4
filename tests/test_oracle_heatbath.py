"""Oracle pins: Creutz SU(2) sampler, Cabibbo-Marinari heat bath and
overrelaxation (Sec. IV.A) against exact densities, the strong- and
weak-coupling limits and exact invariances."""
import numpy as np
import pytest
import scipy.integrate
import scipy.special
import scipy.stats

from _helpers import random_su3, unitarity_violation


@pytest.mark.parametrize("k", [0.5, 2.0, 10.0])
def test_creutz_a0_density_and_acceptance(orc, k):
    n = 400_000
    x, acc = orc.creutz_samples(k, 1234 + int(k * 10), n)
    p_acc = np.pi * scipy.special.i1(k) / (2 * np.sinh(k))
    rate = acc.mean()
    assert abs(rate - p_acc) < 5 * np.sqrt(p_acc * (1 - p_acc) / n)
    a0 = x[acc == 1, 0]
    edges = np.linspace(-1, 1, 41)
    dens = lambda a: np.sqrt(max(0.0, 1 - a * a)) * np.exp(k * (a - 1))
    probs = np.array([scipy.integrate.quad(dens, edges[i], edges[i + 1])[0] for i in range(40)])
    probs /= probs.sum()
    counts, _ = np.histogram(a0, bins=edges)
    mask = probs * a0.size > 20
    exp_c = probs[mask] * a0.size
    chi2 = np.sum((counts[mask] - exp_c) ** 2 / exp_c)
    assert scipy.stats.chi2.sf(chi2, mask.sum() - 1) > 1e-4
    # the accepted element is a unit quaternion with isotropic direction
    xa = x[acc == 1]
    assert np.max(np.abs(np.sum(xa * xa, axis=1) - 1)) < 1e-14
    r2 = 1 - a0 * a0
    for c in (1, 2, 3):
        assert abs(xa[:, c].mean()) < 5 * np.sqrt(r2.mean() / 3 / a0.size)
        assert abs(np.mean(xa[:, c] ** 2) - r2.mean() / 3) < 5 * np.sqrt(np.var(xa[:, c] ** 2) / a0.size)


def test_strong_coupling_plaquette(orc):
    # leading SU(3) character expansion: <W> = beta/18 + beta^2/216 + O(beta^4)
    beta, dims = 0.5, [4, 4, 4, 4]
    U = orc.init_links(dims, 1, seed=2)
    p = orc.update_chain(U, dims, beta, 2, 0, 0, 400, 1, 0)[20:]
    pred = beta / 18 + beta**2 / 216
    assert abs(p.mean() - pred) < 4 * p.std() / np.sqrt(p.size) + 2e-4


def test_weak_coupling_plaquette(orc):
    # leading-order perturbation theory for SU(3), D=4: <1 - W> = 2/beta + O(1/beta^2)
    beta, dims = 100.0, [4, 4, 4, 4]
    U = orc.init_links(dims, 0)
    p = orc.update_chain(U, dims, beta, 3, 0, 0, 150, 1, 2)[50:]
    assert abs((1 - p.mean()) * beta / 2 - 1) < 0.05


def test_heatbath_keeps_su3_and_is_thread_independent(orc):
    dims = [4, 4, 4, 4]
    U1 = orc.init_links(dims, 1, seed=4)
    U2 = U1.copy()
    n0 = orc.get_threads()
    try:
        orc.set_threads(1)
        d1 = orc.new_decisions(dims)
        orc.heatbath_sweep(U1, dims, 5.7, 4, 0, 0, 1, d1)
        orc.set_threads(4)
        d2 = orc.new_decisions(dims)
        orc.heatbath_sweep(U2, dims, 5.7, 4, 0, 0, 1, d2)
    finally:
        orc.set_threads(n0)
    assert np.array_equal(U1, U2) and np.array_equal(d1, d2)
    assert unitarity_violation(U1) < 1e-14
    # with N_hb = 1 the decision is the attempt index 0 or "none" (255)
    assert set(np.unique(d1)) <= {0, 255}


def test_more_attempts_accept_more(orc):
    dims = [4, 4, 4, 4]
    U = orc.init_links(dims, 0)
    orc.update_chain(U, dims, 5.7, 5, 0, 0, 5, 1, 2)
    rates = []
    for n_hb in (1, 4):
        Uc = U.copy()
        d = orc.new_decisions(dims)
        orc.heatbath_sweep(Uc, dims, 5.7, 5, 0, 100, n_hb, d)
        rates.append(np.mean(d != 255))
    assert rates[1] > rates[0] > 0.3


def test_subsweep_equals_sweep_step(orc):
    dims = [4, 2, 4, 2]
    U = orc.init_links(dims, 1, seed=6)
    A = U.copy()
    orc.heatbath_sweep(A, dims, 5.7, 6, 0, 3, 2)
    B = U.copy()
    for mu in range(4):
        for par in range(2):
            orc.heatbath_subsweep(B, dims, 5.7, 6, 0, 3, 2, mu, par)
    assert np.array_equal(A, B)


def test_overrelaxation_preserves_action(orc):
    dims = [4, 4, 4, 4]
    U = orc.init_links(dims, 1, seed=7)
    orc.update_chain(U, dims, 5.7, 7, 0, 0, 5, 1, 0)
    s0 = orc.action(U, dims, 5.7)
    for _ in range(3):
        orc.overrelax_sweep(U, dims)
    assert abs(orc.action(U, dims, 5.7) - s0) < 1e-12 * abs(s0)
    assert unitarity_violation(U) < 1e-14


def test_overrelaxation_local_invariance_and_involution(orc):
    rng = np.random.default_rng(8)
    for _ in range(10):
        Ul = random_su3(rng)
        A = sum(random_su3(rng) for _ in range(6))
        R = orc.or_link_ordered(Ul, A, [0, 1, 2])
        assert abs(np.trace(R @ A).real - np.trace(Ul @ A).real) < 1e-13
        assert np.max(np.abs(R - Ul)) > 1e-3
        back = orc.or_link_ordered(R, A, [2, 1, 0])
        assert np.max(np.abs(back - Ul)) < 1e-13


def test_heatbath_one_link_matches_subsweep(orc):
    dims = [4, 4, 2, 2]
    U = orc.init_links(dims, 1, seed=10)
    B = U.copy()
    dec = orc.new_decisions(dims)
    orc.heatbath_subsweep(B, dims, 6.0, 10, 1, 4, 1, 2, 1, dec)
    for s in range(U.shape[0]):
        x = orc.coords(dims, s)
        if sum(x) % 2 != 1:
            continue
        Un, d = orc.heatbath_one_link(U, dims, 6.0, 10, 1, 4, 1, s, 2)
        assert np.array_equal(Un, B[s, 2]) and np.array_equal(d, dec[s, 2])


def test_heatbath_link_staple_matches_one_link(orc):
    """The lattice-free form (link and staple supplied) is the same map, bit for
    bit; on a cold start every staple is 6 x identity."""
    dims = [4, 2, 4, 2]
    U = orc.init_links(dims, 1, seed=12)
    for s in range(0, U.shape[0], 3):
        for mu in (0, 3):
            ref, dref = orc.heatbath_one_link(U, dims, 6.0, 12, 2, 7, 2, s, mu)
            got, d = orc.heatbath_link_staple(U[s, mu], orc.staple(U, dims, s, mu), 6.0, 12, 2, 7, 2, s, mu)
            assert np.array_equal(got, ref) and np.array_equal(d, dref)
    C = orc.init_links(dims, 0)
    assert np.array_equal(orc.staple(C, dims, 5, 1), 6 * np.eye(3))
    ref, _ = orc.heatbath_one_link(C, dims, 6.0, 12, 0, 1, 1, 5, 1)
    got, _ = orc.heatbath_link_staple(np.eye(3), 6 * np.eye(3), 6.0, 12, 0, 1, 1, 5, 1)
    assert np.array_equal(got, ref)
