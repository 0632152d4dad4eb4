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


# ---------------------------------------------------------------- adaptive step
# Sec. IV.B, Table II: adaptive step (embedded second-order estimate from the
# RK3 stages), tolerance 0.01, maximal step 0.2.


def test_adaptive_error_estimate_is_third_order(orc):
    """d(h) = |W3 - exp(2 Z1 - Z0) W0| is the local error of a second-order
    method: d(h) / d(h/2) -> 8.  A first-order combination (e.g. exp(Z1) W0
    or exp(Z0) W0) gives 4, a wrong stage weight in W3 spoils the ratio."""
    dims = [4, 4, 4, 4]
    U = orc.init_links(dims, 1, seed=3)
    ds = []
    for h in (0.04, 0.02, 0.01):
        W = U.copy()
        ds.append(orc.flow_trial_step(W, dims, h))
    r1, r2 = ds[0] / ds[1], ds[1] / ds[2]
    assert 7.5 < r1 < 8.5 and 7.5 < r2 < 8.5, (ds, r1, r2)
    # the trial step itself is the fixed RK3 step
    W, W2 = U.copy(), U.copy()
    orc.flow_trial_step(W, dims, 0.02)
    orc.flow_step(W2, dims, 0.02)
    assert np.array_equal(W, W2)


def test_adaptive_with_loose_tolerance_is_the_fixed_step_flow(orc):
    """tol so large that every trial is kept and the step pinned at eps_max:
    the same arithmetic as the fixed-step flow (binary-exact step 1/16)."""
    dims = [4, 4, 2, 4]
    U = orc.init_links(dims, 1, seed=4)
    W = U.copy()
    E, Q, steps, rejects = orc.wilson_flow_adaptive(W, dims, 1.0, 1e9, 0.0625, 0.0625, 0.25)
    Wf = U.copy()
    Ef, Qf = orc.wilson_flow(Wf, dims, 0.0625, 16, 4)
    assert (steps, rejects) == (16, 0)
    assert np.array_equal(E, Ef) and np.array_equal(Q, Qf) and np.array_equal(W, Wf)


def _thermal(orc, dims, beta, seed, n):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 4)
    return U


def test_adaptive_matches_fixed_step_flow_within_paper_deviation(orc):
    """Sec. IV.B: with tolerance 0.01 and maximal step 0.2 the adaptive flow's
    E(t) deviated from the fixed-step (0.01) flow by at most about 0.02 % up to
    5 t0 and Q agreed per configuration.  Here: a thermalised 4^3 x 8 field at
    the beta of the 12^3 x 24 ensemble (t0 ~ 0.73), measurements every
    0.18 ~ t0/4.  Smaller tolerances converge to the fixed-step flow."""
    dims, beta = [4, 4, 4, 8], 5.626
    U = _thermal(orc, dims, beta, 11, 60)
    Ef, Qf = orc.wilson_flow(U.copy(), dims, 0.01, 180, 18)
    devs = []
    for tol in (0.01, 1e-3, 1e-4):
        W = U.copy()
        E, Q, steps, rejects = orc.wilson_flow_adaptive(W, dims, 1.8, tol, 0.2, 0.01, 0.18)
        assert len(E) == 11
        devs.append(np.max(np.abs(E - Ef) / Ef))
        assert np.max(np.abs(Q - Qf)) < 2e-3
        assert steps >= 1.8 / 0.2
    assert devs[0] < 2e-4, devs
    assert devs[1] < devs[0] / 3 and devs[2] < devs[1] / 3, devs


def test_adaptive_controller_rejects_and_lands_on_measurement_times(orc):
    """An oversized first trial is rejected and the field restored; the run
    still measures at every k dt_meas <= t_end and at t_end, and agrees with a
    run whose first trial is small."""
    dims = [4, 4, 4, 8]
    U = _thermal(orc, dims, 5.626, 12, 30)
    assert orc.adaptive_measurements(1.0, 0.25) == 5
    assert orc.adaptive_measurements(1.1, 0.25) == 6
    assert orc.adaptive_measurements(0.0, 0.25) == 1
    Wa, Wb = U.copy(), U.copy()
    Ea, Qa, sa, ra = orc.wilson_flow_adaptive(Wa, dims, 1.1, 1e-4, 0.2, 0.2, 0.25)
    Eb, Qb, sb, rb = orc.wilson_flow_adaptive(Wb, dims, 1.1, 1e-4, 0.2, 0.001, 0.25)
    assert ra >= 1 and len(Ea) == len(Eb) == 6
    assert Ea[0] == Eb[0]
    assert np.max(np.abs(Ea - Eb) / Eb) < 1e-5


def test_flow_to_measurement_times(orc):
    """Flow with measurement times (the problem statement's t_meas form): on the
    step grid it reproduces the fixed-step flow bit for bit; off the grid a step
    is shortened to land on the time, which keeps the third-order accuracy."""
    dims = [4, 4, 4, 4]
    U = orc.init_links(dims, 1, seed=31)
    orc.update_chain(U, dims, 6.0, 31, 0, 0, 4, 1, 2)
    W1, W2 = U.copy(), U.copy()
    E1, Q1 = orc.wilson_flow(W1, dims, 0.02, 10, 5)
    E2, Q2 = orc.wilson_flow_times(W2, dims, 0.2, 0.02, [0.0, 0.1, 0.2])
    assert np.array_equal(E1, E2) and np.array_equal(Q1, Q2) and np.array_equal(W1, W2)
    # off-grid times: t = 0.033 and 0.077 with eps = 0.01, against eps = 0.0005
    tm = [0.033, 0.077]
    W3, W4, Wr = U.copy(), U.copy(), U.copy()
    E3, Q3 = orc.wilson_flow_times(W3, dims, 0.1, 0.01, tm)
    E4, Q4 = orc.wilson_flow_times(W4, dims, 0.1, 0.005, tm)
    Er, Qr = orc.wilson_flow_times(Wr, dims, 0.1, 0.0005, tm)
    assert np.max(np.abs(E3 - Er)) < 1e-6 * np.max(np.abs(Er))
    ratio = np.max(np.abs(W3 - Wr)) / np.max(np.abs(W4 - Wr))
    assert 6.0 < ratio < 10.0, ratio  # global error ~ eps^3 with the shortened steps
    # a single step of the whole length is exactly one flow step
    W5, W6 = U.copy(), U.copy()
    orc.wilson_flow_times(W5, dims, 0.037, 1.0, [])
    orc.flow_step(W6, dims, 0.037)
    assert np.array_equal(W5, W6)
    # the improved-charge option measures the improved Q of the flowed field
    W7 = U.copy()
    E7, Q7 = orc.wilson_flow_times(W7, dims, 0.05, 0.01, [0.05], charge=1)
    assert Q7[0] == orc.topo_charge_improved(W7, dims)[0] and E7[0] == orc.clover_EQ(W7, dims)[0]
