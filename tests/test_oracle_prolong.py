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
