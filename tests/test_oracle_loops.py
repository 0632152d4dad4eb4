"""Oracle pins: m x n Wilson loops, partial plaquettes, displaced 2x2 loops and
the smoothness h (Sec. III, IV.C) -- unit gauge, constant-flux closed forms,
the paper's normalisations by brute-force counting, and the exact statement
that after the transfer the 2x2 loops from even sites are the coarse
plaquettes (so W2x2_0 of the fine lattice is the coarse average plaquette)."""
import itertools

import numpy as np

from _helpers import flux_field, gauge_transform, random_su3


def test_unit_gauge_and_plaquette(orc):
    dims = [4, 4, 2, 4]
    U = orc.init_links(dims, 0)
    assert orc.wilson_loop(U, dims, 2, 3) == 1.0
    assert np.allclose(orc.partial_loops(U, dims)[:8], 1.0, atol=0) and orc.partial_loops(U, dims)[8] == 0.0
    U = orc.init_links(dims, 1, seed=2)
    assert abs(orc.wilson_loop(U, dims, 1, 1) - orc.plaquette(U, dims)) < 1e-15


def test_constant_flux_loops(orc):
    dims = [8, 4, 4, 8]
    U, f, g = flux_field(dims, 1, 1)
    for m, n in [(1, 1), (2, 2), (1, 3)]:
        want = ((2 * np.cos(m * n * f) + 1) / 3 + (2 * np.cos(m * n * g) + 1) / 3 + 4) / 6
        assert abs(orc.wilson_loop(U, dims, m, n) - want) < 1e-12


def test_normalisations_count_the_classes(orc):
    # the paper's N_d formulas (Sec. III) equal brute-force counts of the classes
    L, D = 4, 4
    N0 = L**4
    n1 = [0, 0, 0]
    n2 = [0] * 5
    for x in itertools.product(range(L), repeat=4):
        chi = sum(v & 1 for v in x)
        for mu, nu in itertools.combinations(range(4), 2):
            n1[sum(x[r] & 1 for r in range(4) if r not in (mu, nu))] += 1
            n2[chi] += 1
    from math import comb

    for d in range(3):
        assert n1[d] == 2 * (D - d) * (D - d - 1) * comb(D, d) * N0 // 16
    for d in range(5):
        assert n2[d] == comb(D, 2) * comb(D, d) * N0 // 16
    assert sum(n1) == sum(n2) == comb(D, 2) * N0
    # with every plaquette equal, each partial average equals that value
    U, f, g = flux_field([L] * 4, 1, 0)
    out = orc.partial_loops(U, [L] * 4)
    p = orc.plaquette(U, [L] * 4)
    assert abs(np.dot(out[:3], [n / (6 * N0) for n in n1]) - p) < 1e-14


def test_transfer_keeps_coarse_plaquettes_in_W2x2_0(orc):
    dc = [4, 2, 4, 2]
    Uc = orc.init_links(dc, 1, seed=6)
    orc.update_chain(Uc, dc, 5.7, 6, 0, 0, 3, 1, 1)
    for Uf in (orc.transfer(Uc, dc), orc.prolongate(Uc, dc, 0.05, 0.0, 5)[0]):
        out = orc.partial_loops(Uf, [2 * v for v in dc])
        assert abs(out[3] - orc.plaquette(Uc, dc)) < 1e-14
        # 4x2 loops from even sites are the coarse 2x1 loops: the average over class 0 of
        # 2x2 loops is exact; the full-lattice averages differ (not translation invariant)


def test_loops_gauge_invariant_and_h(orc):
    dims = [4, 4, 4, 2]
    U = orc.init_links(dims, 1, seed=8)
    orc.update_chain(U, dims, 5.7, 8, 0, 0, 2, 1, 1)
    g = random_su3(np.random.default_rng(1), U.shape[0])
    Ug = gauge_transform(U, dims, g)
    assert abs(orc.wilson_loop(U, dims, 2, 1) - orc.wilson_loop(Ug, dims, 2, 1)) < 1e-13
    a, b = orc.partial_loops(U, dims), orc.partial_loops(Ug, dims)
    assert np.max(np.abs(a - b)) < 1e-13
    assert 0 < a[8] <= 6.0


def test_plaquette_sum_from_odd_time_links_and_spatial_planes(orc):
    """The decomposition the plaquette-measuring overrelaxation sweep relies
    on (Sec. III plaquette, Sec. IV.A overrelaxation): the plaquettes of the
    planes (3, nu) are the staple products Re Tr(U_3(x) A_3(x)) of the odd
    sites, each counted once, and overrelaxation keeps each such product."""
    dims = [4, 2, 4, 6]
    U = orc.init_links(dims, 1, seed=21)
    V = U.shape[0]
    total = orc.plaquette(U, dims) * 18 * V
    spatial = 0.0
    for s in range(V):
        x = orc.coords(dims, s)
        for mu in range(3):
            for nu in range(mu + 1, 3):
                xm = list(x); xm[mu] = (xm[mu] + 1) % dims[mu]
                xn = list(x); xn[nu] = (xn[nu] + 1) % dims[nu]
                P = U[s, mu] @ U[orc.site_index(dims, xm), nu] @ U[orc.site_index(dims, xn), mu].conj().T @ U[s, nu].conj().T
                spatial += P.trace().real
    odd = [s for s in range(V) if sum(orc.coords(dims, s)) % 2 == 1]
    timelike = sum((U[s, 3] @ orc.staple(U, dims, s, 3)).trace().real for s in odd)
    assert abs(spatial + timelike - total) < 1e-10 * max(1.0, abs(total))
    # overrelaxation of one link leaves its staple product unchanged
    s = odd[3]
    A = orc.staple(U, dims, s, 3)
    new = orc.overrelax_one_link(U, dims, s, 3)
    assert abs((new @ A).trace().real - (U[s, 3] @ A).trace().real) < 1e-12
