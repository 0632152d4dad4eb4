"""Oracle pins: the three-loop improved topological charge (Sec. IV.C; the
gluonic operator of de Forcrand, Garcia Perez and Stamatescu, Nucl. Phys. B
499 (1997) 409): clover charges from m x m leaves, m = 1, 2, 3, combined with
the tree-level coefficients (3/2, -3/5, 1/10)."""
import numpy as np

from _helpers import flux_field, gauge_transform, random_su3


def test_mxm_clover_charges_on_constant_flux(orc):
    # every m x m loop of a constant abelian flux is exp(i m^2 f H), so
    # G_01 = i sin(m^2 f) H and Q_m = V sin(m^2 f) sin(m^2 g) / (2 pi^2) exactly
    for dims, n01, n23 in (([8, 8, 8, 8], 1, 1), ([8, 6, 10, 8], 2, -1)):
        U, f, g = flux_field(dims, n01, n23)
        V = int(np.prod(dims))
        q = orc.topo_charge_improved(U, dims)
        for m in (1, 2, 3):
            want = V * np.sin(m * m * f) * np.sin(m * m * g) / (2 * np.pi**2)
            assert abs(q[m] - want) < 1e-10 * max(1.0, abs(want)), (m, q[m], want)
        assert abs(q[0] - (1.5 * q[1] - 0.6 * q[2] / 16 + 0.1 * q[3] / 81)) < 1e-12
        # the 1 x 1 charge is the clover charge
        assert abs(q[1] - orc.clover_EQ(U, dims)[1]) < 1e-11


def test_improved_charge_approaches_the_integer_faster(orc):
    # constant flux, Q_cont = 2 n01 n23: the clover error falls as f^2 ~ L^-4,
    # the improved one as f^4 ~ L^-8
    errs = {}
    for L in (8, 12, 16):
        U, f, g = flux_field([L] * 4, 1, 1)
        q = orc.topo_charge_improved(U, [L] * 4)
        errs[L] = (abs(q[1] - 2), abs(q[0] - 2))
    for a, b in ((8, 12), (12, 16)):
        r = b / a
        assert 0.8 * r**4 < errs[a][0] / errs[b][0] < 1.25 * r**4
        assert 0.7 * r**8 < errs[a][1] / errs[b][1] < 1.4 * r**8
    assert errs[16][1] < 0.1 * errs[16][0]


def _smooth_abelian(L, amp0=3.0, amp2=2.0, L1=8, L3=8):
    """Links diag(e^{i t}, e^{-i t}, 1) of the periodic continuum potential
    A_1 = amp0 sin(2 pi y0) / (2 pi), A_3 = amp2 sin(2 pi y2) / (2 pi) on a
    unit torus sampled with spacing a = 1/L in directions 0 and 2 (the field
    does not depend on y1, y3).  Link phases are the exact line integrals, so
    every loop is the exponential of the flux through it.  F_01 = amp0 cos(2 pi y0),
    F_23 = amp2 cos(2 pi y2); continuum density q = F_01 F_23 / (2 pi^2)."""
    dims = [L, L1, L, L3]
    V = int(np.prod(dims))
    s = np.arange(V)
    x0, x2 = s % L, (s // (L * L1)) % L
    a = 1.0 / L
    th = np.zeros((V, 4))
    th[:, 1] = a * amp0 * np.sin(2 * np.pi * x0 * a) / (2 * np.pi)
    th[:, 3] = a * amp2 * np.sin(2 * np.pi * x2 * a) / (2 * np.pi)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = np.exp(1j * th)
    U[:, :, 1, 1] = np.exp(-1j * th)
    U[:, :, 2, 2] = 1
    return U, dims


def test_improved_density_is_accurate_to_order_a6(orc):
    # at a fixed physical point the m x m clover densities differ from the
    # continuum by (m a)^2 terms; the improved combination only at O(a^6):
    # halving a divides the clover error by 4 and the improved one by 64
    def errors(L):
        U, dims = _smooth_abelian(L)
        y0, y2 = 1 / 8, 3 / 8
        s = int(round(y0 * L)) + dims[0] * dims[1] * int(round(y2 * L))
        cont = 3.0 * np.cos(2 * np.pi * y0) * 2.0 * np.cos(2 * np.pi * y2) / (2 * np.pi**2)
        clover = orc.clover_q_site(U, dims, s, 1) * L**4
        imp = orc.clover_q_site(U, dims, s, 0) * L**4
        return abs(clover - cont), abs(imp - cont)

    e = {L: errors(L) for L in (16, 32, 64)}
    for a, b in ((16, 32), (32, 64)):
        assert 3.5 < e[a][0] / e[b][0] < 4.5, (e[a], e[b])
        assert 45 < e[a][1] / e[b][1] < 90, (e[a], e[b])


def test_improved_charge_is_gauge_invariant(orc):
    dims = [4, 4, 4, 6]
    U = orc.init_links(dims, 1, seed=21)
    orc.update_chain(U, dims, 6.0, 21, 0, 0, 3, 1, 2)
    g = random_su3(np.random.default_rng(22), U.shape[0])
    a = orc.topo_charge_improved(U, dims)
    b = orc.topo_charge_improved(gauge_transform(U, dims, g), dims)
    assert np.max(np.abs(a - b)) < 1e-11
    assert abs(a[0]) > 1e-3  # the invariance is not vacuous
