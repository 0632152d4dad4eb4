"""Oracle pins: Wilson flow (Sec. IV.B; Luscher's third-order Runge-Kutta
integrator) -- heat-kernel decay of an abelian plane wave (smoothing radius
sqrt(8t)), third-order convergence, monotone action, gauge covariance."""
import numpy as np

from _helpers import gauge_transform, random_su3


def test_plane_wave_decays_with_lattice_laplacian(orc):
    dims = [8, 2, 2, 2]
    V = 64
    amp, eps, nsteps = 1e-3, 0.01, 50
    U = orc.init_links(dims, 0)
    p = 2 * np.pi / dims[0]
    th = np.zeros(V)
    for s in range(V):
        x0 = orc.coords(dims, s)[0]
        th[s] = amp * np.cos(p * x0)
        U[s, 1] = np.diag(np.exp(1j * th[s] * np.array([1.0, -1.0, 0.0])))
    for _ in range(nsteps):
        orc.flow_step(U, dims, eps)
    t = eps * nsteps
    th_t = np.angle(U[:, 1, 0, 0])
    ratio = np.dot(th_t, th) / np.dot(th, th)
    phat2 = 4 * np.sin(p / 2) ** 2
    assert abs(ratio / np.exp(-phat2 * t) - 1) < 1e-5


def test_flow_is_third_order(orc):
    dims = [4, 4, 2, 2]
    U0 = orc.init_links(dims, 1, seed=1)
    orc.update_chain(U0, dims, 6.0, 1, 0, 0, 5, 1, 1)
    t = 0.2

    def run(eps):
        W = U0.copy()
        for _ in range(int(round(t / eps))):
            orc.flow_step(W, dims, eps)
        return W

    ref = run(0.2 / 64)
    errs = [np.max(np.abs(run(e) - ref)) for e in (0.05, 0.025, 0.0125)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 6.5 < r1 < 9.5 and 6.5 < r2 < 9.5, (errs, r1, r2)


def test_flow_increases_plaquette_and_is_covariant(orc):
    dims = [4, 4, 4, 2]
    U = orc.init_links(dims, 1, seed=2)
    orc.update_chain(U, dims, 6.0, 2, 0, 0, 5, 1, 1)
    rng = np.random.default_rng(3)
    g = random_su3(rng, U.shape[0])
    Ug = gauge_transform(U, dims, g)
    E, Q = orc.wilson_flow(U, dims, 0.02, 10, 2)
    Eg, Qg = orc.wilson_flow(Ug, dims, 0.02, 10, 2)
    # clover E is not the flowed action and may rise at the very first steps of a rough field
    assert E[-1] < 0.9 * E[0]
    assert np.max(np.abs(E - Eg)) < 1e-12 and np.max(np.abs(Q - Qg)) < 1e-12
    assert np.max(np.abs(gauge_transform(U, dims, g) - Ug)) < 1e-12
    W = U.copy()
    p = [orc.plaquette(W, dims)]
    for _ in range(5):
        orc.flow_step(W, dims, 0.02)
        p.append(orc.plaquette(W, dims))
    assert np.all(np.diff(p) > 0)


def test_flow_keeps_constant_flux_fixed(orc):
    # a constant abelian field strength is a stationary point of the Wilson action
    from _helpers import flux_field

    dims = [4, 4, 4, 4]
    U, f, g = flux_field(dims, 1, 1)
    E0, Q0 = orc.clover_EQ(U, dims)
    W = U.copy()
    for _ in range(3):
        orc.flow_step(W, dims, 0.05)
    E1, Q1 = orc.clover_EQ(W, dims)
    assert abs(E1 - E0) < 1e-12 and abs(Q1 - Q0) < 1e-11
