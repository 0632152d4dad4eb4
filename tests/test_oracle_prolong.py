"""Oracle pins: restriction, transfer and APE interpolation (Sec. III,
Eqs. restriction, prolongation, smoothing, APE; Sec. IV.C)."""
import numpy as np

from _helpers import unitarity_violation


def _coarse(orc, dims_c, beta=5.7, seed=1, n=4):
    U = orc.init_links(dims_c, 1, seed=seed)
    orc.update_chain(U, dims_c, beta, seed, 0, 0, n, 1, 2)
    return U


def _loop(U, dims, s, path):
    """Product of links along a path of (mu, +1/-1) steps starting at site s."""
    L = [int(v) for v in dims]
    x = [(s // int(np.prod(L[:m]))) % L[m] for m in range(4)]
    M = np.eye(3, dtype=np.complex128)
    for mu, d in path:
        if d > 0:
            idx = x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))
            M = M @ U[idx, mu]
            x[mu] = (x[mu] + 1) % L[mu]
        else:
            x[mu] = (x[mu] - 1) % L[mu]
            idx = x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))
            M = M @ U[idx, mu].conj().T
    return M


def _rect(mu, nu, m, n):
    return [(mu, 1)] * m + [(nu, 1)] * n + [(mu, -1)] * m + [(nu, -1)] * n


def test_restriction_inverts_transfer_exactly(orc):
    dc = [2, 4, 2, 4]
    Uc = _coarse(orc, dc)
    Uf = orc.transfer(Uc, dc)
    assert np.array_equal(orc.restrict(Uf, [2 * v for v in dc]), Uc)
    Uf2, iters, _ = orc.prolongate(Uc, dc, 0.05, 0.0, 5)
    assert iters == [5, 5, 5]
    assert np.array_equal(orc.restrict(Uf2, [2 * v for v in dc]), Uc)


def test_transferred_bonds_unchanged_and_all_bonds_su3(orc):
    dc = [2, 2, 4, 2]
    df = [2 * v for v in dc]
    Uc = _coarse(orc, dc, seed=2)
    Uf0 = orc.transfer(Uc, dc)
    Uf, iters, _ = orc.prolongate(Uc, dc, 0.05, 1e-5, 2000)
    assert unitarity_violation(Uf) < 1e-13
    for s in range(Uf.shape[0]):
        x = orc.coords(df, s)
        for mu in range(4):
            if all(x[nu] % 2 == 0 for nu in range(4) if nu != mu):  # chi_mu = 0
                assert np.array_equal(Uf[s, mu], Uf0[s, mu])
                want = np.eye(3) if x[mu] % 2 else Uc[orc.site_index(dc, [v // 2 for v in x]), mu]
                assert np.array_equal(Uf[s, mu], want)
            else:
                assert np.max(np.abs(Uf0[s, mu] - np.eye(3))) == 0.0


def test_even_site_loops_equal_coarse_loops(orc):
    # 2m x 2n loops from even fine sites equal m x n coarse loops (exactly preserved by the map)
    dc = [4, 2, 2, 4]
    df = [2 * v for v in dc]
    Uc = _coarse(orc, dc, seed=3)
    Uf, _, _ = orc.prolongate(Uc, dc, 0.05, 0.0, 20)
    for sc in range(0, Uc.shape[0], 3):
        xc = orc.coords(dc, sc)
        sf = orc.site_index(df, [2 * v for v in xc])
        for mu in range(4):
            for nu in range(mu + 1, 4):
                for (m, n) in [(1, 1), (1, 2)]:
                    wc = np.trace(_loop(Uc, dc, sc, _rect(mu, nu, m, n))).real
                    wf = np.trace(_loop(Uf, df, sf, _rect(mu, nu, 2 * m, 2 * n))).real
                    assert abs(wc - wf) < 1e-13


def test_interpolation_lowers_each_partial_action(orc):
    dc = [2, 2, 2, 4]
    df = [2 * v for v in dc]
    Uc = _coarse(orc, dc, seed=4)
    Uf0 = orc.transfer(Uc, dc)
    before = [orc.partial_action(Uf0, df, d) for d in range(3)]
    Uf, iters, sd = orc.prolongate(Uc, dc, 0.05, 1e-5, 5000)
    assert all(1 < it < 5000 for it in iters), iters
    # stage d minimises S_d over its active bonds, starting from the transfer
    assert sd[0] < before[0]
    # the final S_d values reported equal a recomputation on the output field
    assert abs(sd[2] - orc.partial_action(Uf, df, 2)) < 1e-12 * max(1, abs(sd[2]))
    # S_d decreases monotonically over the APE iterations of a stage (checked for d = 0)
    vals = []
    for n in (1, 2, 4, 8, 16):
        U1, _, s1 = orc.prolongate(Uc, dc, 0.05, 0.0, n)
        vals.append(orc.partial_action(U1, df, 0))
    assert all(b <= a + 1e-12 for a, b in zip(vals, vals[1:])), vals


def test_stage_stopping_rule(orc):
    dc = [2, 2, 2, 2]
    Uc = _coarse(orc, dc, seed=5)
    _, it_loose, _ = orc.prolongate(Uc, dc, 0.05, 1e-3, 10000)
    _, it_tight, _ = orc.prolongate(Uc, dc, 0.05, 1e-6, 10000)
    assert all(a < b for a, b in zip(it_loose, it_tight))


def test_cold_coarse_prolongates_to_cold_fine(orc):
    dc = [2, 2, 2, 2]
    Uc = orc.init_links(dc, 0)
    Uf, iters, sd = orc.prolongate(Uc, dc, 0.05, 1e-5, 100)
    assert np.max(np.abs(Uf - np.eye(3))) < 1e-15 and np.all(sd == 0)


# ---- one Jacobi APE step of stage d (Eq. APE), pinned without the prolongation around it

def _pure_gauge(dims, rng):
    from _helpers import gauge_transform, random_su3

    V = int(np.prod(dims))
    g = random_su3(rng, V)
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    return gauge_transform(one, dims, g)


def test_ape_step_fixes_pure_gauge_fields(orc):
    # On U_mu(n) = g(n) g(n+mu)^+ every staple T+/- equals U_mu(n), so the smeared
    # sum is (1 + 2(d+1)c) U and projects back onto U.  A staple with a misplaced
    # dagger (e.g. the printed T- with U_nu(n-nu+mu)^+) breaks this.
    rng = np.random.default_rng(11)
    for dims in ([4, 4, 4, 6], [2, 4, 6, 4]):
        U = _pure_gauge(dims, rng)
        for d in range(3):
            assert np.max(np.abs(orc.ape_step(U, dims, d) - U)) < 1e-14


def test_ape_step_is_gauge_covariant(orc):
    # APE(g U g^+) = g APE(U) g^+ for a random local g(n).  The projection is
    # covariant at its maximiser; 30 passes converge it far below the bar.
    from _helpers import gauge_transform, random_su3

    rng = np.random.default_rng(12)
    dims = [4, 4, 4, 6]
    U = orc.init_links(dims, 1, seed=3)
    orc.update_chain(U, dims, 5.7, 3, 0, 0, 2, 1, 1)
    g = random_su3(rng, U.shape[0])
    for d in range(3):
        lhs = gauge_transform(orc.ape_step(U, dims, d, n_pass=30), dims, g)
        rhs = orc.ape_step(gauge_transform(U, dims, g), dims, d, n_pass=30)
        assert np.max(np.abs(lhs - rhs)) < 1e-12
        # the step does move the field (the covariance is not vacuous)
        assert np.max(np.abs(orc.ape_step(U, dims, d) - U)) > 1e-2


def _u1_ape(theta, dims, d, c):
    """Abelian APE step on link angles theta[x0,x1,x2,x3,mu] (U(1) smearing, written
    with phases): active bonds have d+1 odd coordinates other than n_mu; the staples
    run in the directions nu != mu with n_nu odd."""
    L = list(dims)
    out = theta.copy()
    sh = lambda a, nu, k: np.roll(a, -k, axis=nu)  # a(n + k e_nu)
    grid = np.indices(L)
    for mu in range(4):
        odd = [grid[nu] % 2 for nu in range(4)]
        chi = sum(odd[nu] for nu in range(4) if nu != mu)
        z = np.exp(1j * theta[..., mu])
        for nu in range(4):
            if nu == mu:
                continue
            tn, tm = theta[..., nu], theta[..., mu]
            up = tn + sh(tm, nu, 1) - sh(tn, mu, 1)
            dn = -sh(tn, nu, -1) + sh(tm, nu, -1) + sh(sh(tn, nu, -1), mu, 1)
            z = z + c * odd[nu] * (np.exp(1j * up) + np.exp(1j * dn))
        act = chi == d + 1
        out[..., mu] = np.where(act, np.angle(z), theta[..., mu])
    return out


def test_ape_step_on_abelian_fields_is_u1_smearing(orc):
    # Links diag(e^{i theta}, e^{-i theta}, 1): the smeared sum stays diag(z, z*, r)
    # with r > 0, whose SU(3) projection is diag(z/|z|, z*/|z|, 1), so the step is
    # the U(1) APE step on theta.  This fixes the active bonds, the staple
    # directions and the sign of c.
    rng = np.random.default_rng(13)
    dims = [4, 2, 6, 4]
    V = int(np.prod(dims))
    theta = rng.uniform(-np.pi, np.pi, size=(dims[3], dims[2], dims[1], dims[0], 4))
    th = np.transpose(theta, (3, 2, 1, 0, 4))  # index [x0,x1,x2,x3,mu]
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    flat = theta.reshape(V, 4)  # x0 fastest matches the canonical site order
    for k, sgn in ((0, 1), (1, -1)):
        U[:, :, k, k] = np.exp(1j * sgn * flat)
    U[:, :, 2, 2] = 1
    for d in range(3):
        ref = np.transpose(_u1_ape(th, dims, d, 0.05), (3, 2, 1, 0, 4)).reshape(V, 4)
        W = orc.ape_step(U, dims, d)
        assert np.max(np.abs(W[:, :, 0, 0] - np.exp(1j * ref))) < 1e-14
        assert np.max(np.abs(W[:, :, 1, 1] - np.exp(-1j * ref))) < 1e-14
        assert np.max(np.abs(W[:, :, 2, 2] - 1)) < 1e-14
