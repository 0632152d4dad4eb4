"""Oracle pins: plaquette, action, staples, force and clover observables
against the unit gauge, gauge invariance/covariance, the staple identity and
closed forms for a constant abelian flux (Sec. III; Sec. IV.B-C)."""
import numpy as np

from _helpers import flux_field, gauge_transform, random_su3

D4 = [4, 4, 4, 4]


def test_unit_gauge(orc):
    U = orc.init_links(D4, 0)
    assert orc.plaquette(U, D4) == 1.0
    assert orc.action(U, D4, 6.0) == 0.0
    assert np.max(np.abs(orc.force(U, D4, 6.0))) == 0.0
    E, Q = orc.clover_EQ(U, D4)
    assert E == 0.0 and Q == 0.0


def test_hot_start_is_su3_and_decorrelated(orc):
    U = orc.init_links(D4, 1, seed=3)
    from _helpers import unitarity_violation

    assert unitarity_violation(U) < 1e-14
    # Haar average of Re Tr U_p / 3 is zero; std of one plaquette is 1/sqrt(18)
    assert abs(orc.plaquette(U, D4)) < 5 / np.sqrt(18 * 6 * 256)


def test_gauge_invariance_and_force_covariance(orc):
    rng = np.random.default_rng(11)
    dims = [4, 4, 2, 4]
    U = orc.init_links(dims, 1, seed=1)
    orc.update_chain(U, dims, 5.7, 1, 0, 0, 3, 1, 1)
    V = U.shape[0]
    g = random_su3(rng, V)
    Ug = gauge_transform(U, dims, g)
    assert abs(orc.plaquette(Ug, dims) - orc.plaquette(U, dims)) < 1e-14
    E0, Q0 = orc.clover_EQ(U, dims)
    E1, Q1 = orc.clover_EQ(Ug, dims)
    assert abs(E1 - E0) < 1e-12 and abs(Q1 - Q0) < 1e-12
    F = orc.force(U, dims, 5.7)
    Fg = orc.force(Ug, dims, 5.7)
    for s in range(0, V, 7):
        for mu in range(4):
            Fm = orc.alg_to_mat(F[s, mu])
            assert np.max(np.abs(orc.alg_to_mat(Fg[s, mu]) - g[s] @ Fm @ g[s].conj().T)) < 1e-12


def test_staple_identity(orc):
    # each plaquette contains four links: sum_{x,mu} Re Tr(U A) = 4 sum_p Re Tr U_p
    dims = [2, 4, 2, 4]
    U = orc.init_links(dims, 1, seed=9)
    V = U.shape[0]
    tot = sum(np.trace(U[s, mu] @ orc.staple(U, dims, s, mu)).real for s in range(V) for mu in range(4))
    assert abs(tot - 4 * 18 * V * orc.plaquette(U, dims)) < 1e-10


def test_constant_flux_closed_forms(orc):
    dims = [4, 6, 4, 8]
    U, f, g = flux_field(dims, 1, 2)
    V = U.shape[0]
    plaq = ((2 * np.cos(f) + 1) + (2 * np.cos(g) + 1) + 12) / 18
    assert abs(orc.plaquette(U, dims) - plaq) < 1e-12
    E, Q = orc.clover_EQ(U, dims)
    assert abs(E - 2 * (np.sin(f) ** 2 + np.sin(g) ** 2)) < 1e-12
    assert abs(Q - V * np.sin(f) * np.sin(g) / (2 * np.pi**2)) < 1e-11
    # the continuum value 2 n01 n23 up to the (sin x / x)^2 lattice factor
    assert abs(Q - 2 * 1 * 2) < 0.15
    # the partial actions split the (0,1) and (2,3) plaquettes as the classification fixes:
    # a (mu,nu) plaquette has chi_munu = number of odd coordinates in the two other directions
    per = (1 - (2 * np.cos(f) + 1) / 3) + (1 - (2 * np.cos(g) + 1) / 3)
    sd = [orc.partial_action(U, dims, d) for d in range(3)]
    assert np.allclose(sd, [V / 4 * per, V / 2 * per, V / 4 * per], rtol=1e-12, atol=1e-12)
    assert abs(sum(sd) - 6 * V * (1 - orc.plaquette(U, dims))) < 1e-10
