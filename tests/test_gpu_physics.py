"""Statistical pins of the GPU path against numbers the paper prints and
against ensembles from the oracle.

* t0/a^2 of the 12^3 x 24, beta = 5.626 ensemble (Table I): heat bath +
  overrelaxation, Wilson flow (fixed step 0.01), clover E, t^2 E(t0) = 0.3 by
  linear interpolation (Sec. IV.B).
* HMC acceptance on the same ensemble at 1/dtau = 37 unit-trajectory steps
  (Table VI) against the model P_acc = erfc(Omega^{1/2} dtau^2 / 2) (App. A).
* GPU and oracle ensembles (independent chains, same action): average
  plaquette and topological susceptibility agree within 2 sigma.
"""
import os

import numpy as np
import pytest
import scipy.special
import torch

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def _gold():
    t0, hmc = {}, {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "t0":
            t0[f[1]] = (float(f[2]), float(f[3]), float(f[4]))
        elif f[0] == "hmc":
            hmc[f[1]] = (float(f[2]), float(f[3]), float(f[4]), int(f[5]))
    return t0, hmc


def _t0_from_flow(E, eps):
    t = eps * np.arange(E.size)
    y = t * t * E
    k = int(np.argmax(y >= 0.3))
    assert k > 0 and y[k] >= 0.3, "flow did not reach t^2 E = 0.3"
    return t[k - 1] + (0.3 - y[k - 1]) * (t[k] - t[k - 1]) / (y[k] - y[k - 1])


def _copy(gpu, lat):
    c = gpu.Lattice(lat.dims, lat.prec, seed=lat.seed, lattice_id=lat.lattice_id)
    c.links.copy_(lat.links)
    return c


@pytest.fixture(scope="module")
def ensemble_12x24(gpu):
    t0_tab, _ = _gold()
    dims = [12, 12, 12, 24]
    beta = t0_tab["12x12x12x24"][0]
    lat = gpu.Lattice(dims, "f32c12", seed=2024, with_mom=True)
    gpu.mgq_init_links(lat, 1)
    gpu.mgq_update_sweeps(lat, beta, 0, 300, 1, 4)
    return lat, beta


def test_t0_matches_table_I(gpu, ensemble_12x24):
    t0_tab, _ = _gold()
    _, t0_paper, t0_err = t0_tab["12x12x12x24"]
    lat, beta = ensemble_12x24
    eps, n_cfg, sep = 0.01, 64, 20
    vals = []
    for i in range(n_cfg):
        gpu.mgq_update_sweeps(lat, beta, 1000 + i * sep, sep, 1, 4)
        w = _copy(gpu, lat)
        E, _ = gpu.mgq_wilson_flow(w, eps, 100, 1)
        vals.append(_t0_from_flow(E, eps))
    vals = np.array(vals)
    mean, err = vals.mean(), vals.std(ddof=1) / np.sqrt(vals.size) * 1.5  # 1.5: autocorrelation allowance
    assert abs(mean - t0_paper) < 3 * np.hypot(err, t0_err), (mean, err, t0_paper)


def test_hmc_acceptance_matches_table_VI(gpu, ensemble_12x24):
    t0_tab, hmc_tab = _gold()
    _, t0, _ = t0_tab["12x12x12x24"]
    omega_t0, omega_err, _, steps = hmc_tab["12x12x12x24"]
    lat, beta = ensemble_12x24
    w = _copy(gpu, lat)
    w.mom = torch.zeros_like(lat.mom)
    w.c.mom = w.mom.data_ptr()
    dtau = 1.0 / steps
    dHs, accs = [], []
    for traj in range(160):
        dH, acc = gpu.mgq_hmc_trajectory(w, beta, 1.0, steps, traj, 1)
        dHs.append(dH)
        accs.append(acc)
    dHs, accs = np.array(dHs[10:]), np.array(accs[10:])
    # Creutz equality on the GPU chain
    ex = np.exp(-dHs)
    assert abs(ex.mean() - 1) < 4 * ex.std(ddof=1) / np.sqrt(ex.size) + 0.02
    # acceptance vs erfc(Omega^{1/2} dtau^2 / 2) with Omega^{1/2} = (Omega^{1/2}/t0) t0 (App. A, Table VI)
    pred = scipy.special.erfc(0.5 * omega_t0 * t0 * dtau**2)
    band = abs(scipy.special.erfc(0.5 * (omega_t0 + 2 * omega_err) * t0 * dtau**2) - pred)
    sig = np.sqrt(pred * (1 - pred) / accs.size) * 1.5
    assert abs(accs.mean() - pred) < 3 * sig + band, (accs.mean(), pred)


def test_gpu_and_oracle_ensembles_agree(gpu, orc):
    """Independent GPU (FP32 12-real) and oracle (FP64) chains on 8^4 at beta = 5.7:
    <W> and chi = <Q^2>/V at flow time t = 1 agree within 2 sigma (errors from
    blocks of 10 configurations)."""
    dims, beta, n_cfg, sep = [8, 8, 8, 8], 5.7, 150, 4
    V = 8**4
    U = orc.init_links(dims, 1, seed=77)
    orc.update_chain(U, dims, beta, 77, 0, 0, 100, 1, 4)
    lat = gpu.Lattice(dims, "f32c12", seed=78)
    gpu.mgq_init_links(lat, 1)
    gpu.mgq_update_sweeps(lat, beta, 0, 100, 1, 4)
    pw, pq, gw, gq = [], [], [], []
    for i in range(n_cfg):
        pw.append(orc.update_chain(U, dims, beta, 77, 0, 200 + i * sep, sep, 1, 4)[-1])
        E, Q = orc.wilson_flow(U.copy(), dims, 0.02, 50, 50)
        pq.append(Q[-1])
        gw.append(gpu.mgq_update_sweeps(lat, beta, 200 + i * sep, sep, 1, 4, plaq_out=True)[-1])
        w = _copy(gpu, lat)
        E, Q = gpu.mgq_wilson_flow(w, 0.02, 50, 50)
        gq.append(Q[-1])
    pw, gw, pq, gq = map(np.array, (pw, gw, pq, gq))

    def blocked(a):
        b = a.reshape(-1, 10).mean(axis=1)
        return a.mean(), b.std(ddof=1) / np.sqrt(b.size)

    for a, b in [(pw, gw), (pq**2 / V, gq**2 / V)]:
        (ma, ea), (mb, eb) = blocked(a), blocked(b)
        assert abs(ma - mb) < 2 * np.hypot(ea, eb), (ma, mb, np.hypot(ea, eb))
