"""GPU parity of the checkerboard heat bath and overrelaxation (Sec. IV.A),
start configurations and plaquette against the FP64 oracle, through the C ABI.

FP64 path: every link within 1e-12 and identical accept/reject decisions.
FP32 paths: plaquette and action within 1e-6 relative after one sweep."""
import numpy as np
import pytest
import torch

from _helpers import unitarity_violation

pytestmark = pytest.mark.gpu

DIMS = [
    [8, 8, 8, 8],     # config-1 lattice: 16 blocks of 128 per sub-sweep
    [6, 6, 6, 6],     # ragged: V/2 = 648 is not a multiple of the block size
    [2, 2, 2, 2],     # degenerate: x+nu and x-nu coincide
    [4, 2, 6, 8],     # anisotropic
]


def _lat(gpu, dims, prec="f64", seed=0, lid=0, **kw):
    return gpu.Lattice(dims, prec, seed=seed, lattice_id=lid, **kw)


def test_hot_start_matches_oracle(gpu, orc):
    dims = [4, 6, 4, 2]
    ref = orc.init_links(dims, 1, seed=17, lattice_id=3)
    lat = _lat(gpu, dims, seed=17, lid=3)
    gpu.mgq_init_links(lat, 1)
    U = lat.to_numpy()
    assert np.max(np.abs(U - ref)) < 1e-13
    gpu.mgq_init_links(lat, 0)
    assert np.array_equal(lat.to_numpy(), orc.init_links(dims, 0))


@pytest.mark.parametrize("prec,tol", [("f64", 0.0), ("f32", 1e-7), ("f32c12", 1e-6)])
def test_import_export_roundtrip(gpu, orc, prec, tol):
    dims = [6, 4, 2, 4]
    ref = orc.init_links(dims, 1, seed=5)
    lat = _lat(gpu, dims, prec)
    lat.from_numpy(ref)
    assert np.max(np.abs(lat.to_numpy() - ref)) <= tol


@pytest.mark.parametrize("dims", DIMS)
def test_heatbath_subsweeps_bit_for_bit_decisions(gpu, orc, dims):
    beta, seed, lid, sweep, n_hb = 5.7, 11, 2, 7, 2
    U = orc.init_links(dims, 1, seed=seed, lattice_id=lid)
    lat = _lat(gpu, dims, seed=seed, lid=lid)
    lat.from_numpy(U)
    V = U.shape[0]
    for mu in range(4):
        for par in range(2):
            dref = orc.new_decisions(dims)
            orc.heatbath_subsweep(U, dims, beta, seed, lid, sweep, n_hb, mu, par, dref)
            dgpu = torch.full((V * 12,), 255, dtype=torch.uint8, device="cuda")
            gpu.mgq_heatbath_subsweep(lat, beta, sweep, n_hb, mu, par, dgpu)
            assert np.array_equal(dgpu.cpu().numpy().reshape(V, 4, 3), dref), (mu, par)
            G = lat.to_numpy()
            assert np.max(np.abs(G - U)) < 1e-12, (mu, par, np.max(np.abs(G - U)))


@pytest.mark.parametrize("dims", DIMS[:2])
def test_overrelaxation_sweep_parity(gpu, orc, dims):
    U = orc.init_links(dims, 1, seed=4)
    orc.update_chain(U, dims, 5.7, 4, 0, 0, 2, 1, 0)
    lat = _lat(gpu, dims)
    lat.from_numpy(U)
    orc.overrelax_sweep(U, dims)
    gpu.mgq_overrelax_sweep(lat)
    # one sweep: within 1e-12 (measured worst 1.3e-13 on hot starts).  Later
    # sweeps amplify the rounding differences (FMA contraction, summation order)
    # through the 1/|w| of the reflection, about x20-x100 per sweep.
    assert np.max(np.abs(lat.to_numpy() - U)) < 1e-12


def test_config1_chain_fp64(gpu, orc):
    """8^4, beta = 5.7, cold start, Philox seed 0, 20 x (1 HB + 4 OR), FP64.

    Two chains that differ by rounding diverge exponentially (about x10 per
    compound sweep at this coupling), so the chain is checked step by step:
    every compound sweep starts on the GPU from the oracle's configuration and
    must reproduce the oracle's next configuration (1e-11), its accept/reject
    decisions (identical) and its plaquette (1e-12)."""
    dims, beta = [8, 8, 8, 8], 5.7
    U = orc.init_links(dims, 0)
    lat = _lat(gpu, dims)
    gpu.mgq_init_links(lat, 0)
    assert np.array_equal(lat.to_numpy(), U)
    V = U.shape[0]
    dgpu = torch.full((V * 12,), 255, dtype=torch.uint8, device="cuda")
    worst = 0.0
    for sweep in range(20):
        lat.from_numpy(U)
        dref = orc.new_decisions(dims)
        orc.heatbath_sweep(U, dims, beta, 0, 0, sweep, 1, dref)
        for _ in range(4):
            orc.overrelax_sweep(U, dims)
        for mu in range(4):
            for par in range(2):
                gpu.mgq_heatbath_subsweep(lat, beta, sweep, 1, mu, par, dgpu)
        for _ in range(4):
            gpu.mgq_overrelax_sweep(lat)
        assert np.array_equal(dgpu.cpu().numpy().reshape(V, 4, 3), dref), sweep
        err = np.max(np.abs(lat.to_numpy() - U))
        worst = max(worst, err)
        assert err < 1e-11, (sweep, err)
        assert abs(gpu.mgq_plaquette(lat) - orc.plaquette(U, dims)) < 1e-12
    assert gpu.mgq_check_unitarity(lat) < 1e-13


def _tau_int(x, c=6.0):
    """Integrated autocorrelation time with automatic windowing (Madras and
    Sokal, J. Stat. Phys. 50 (1988) 109): the first window W >= c tau(W)."""
    y = np.asarray(x, dtype=np.float64) - np.mean(x)
    n = y.size
    f = np.fft.rfft(y, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n]
    acf = acf / acf[0]
    tau = 0.5
    for w in range(1, n // 2):
        tau += acf[w]
        if w >= c * tau:
            break
    return max(tau, 0.5)


def test_config1_free_chain_statistics(gpu, orc):
    """The free-running GPU chain and the oracle chain (same seed, 8^4, beta =
    5.7, cold start) agree in distribution: mean plaquette over sweeps 20..119
    within 3 combined sigma, each error from the chain's own integrated
    autocorrelation time (var * 2 tau_int / n)."""
    dims, beta, n = [8, 8, 8, 8], 5.7, 120
    U = orc.init_links(dims, 0)
    pref = orc.update_chain(U, dims, beta, 0, 0, 0, n, 1, 4)
    lat = _lat(gpu, dims)
    gpu.mgq_init_links(lat, 0)
    pg = gpu.mgq_update_sweeps(lat, beta, 0, n, 1, 4, plaq_out=True)
    assert np.max(np.abs(pg[:3] - pref[:3])) < 1e-12  # early sweeps still agree link by link
    a, b = pref[20:], pg[20:]
    err = [np.sqrt(v.var(ddof=1) * 2 * _tau_int(v) / v.size) for v in (a, b)]
    assert abs(a.mean() - b.mean()) < 3 * np.hypot(*err), (a.mean(), b.mean(), err)


@pytest.mark.parametrize("prec", ["f32", "f32c12"])
def test_fp32_one_sweep_plaquette_and_action(gpu, orc, prec):
    dims, beta = [16, 16, 16, 16], 6.0
    U = orc.init_links(dims, 1, seed=8)
    orc.update_chain(U, dims, beta, 8, 0, 0, 3, 1, 1)
    lat = _lat(gpu, dims, prec, seed=8)
    lat.from_numpy(U)
    orc.update_chain(U, dims, beta, 8, 0, 3, 1, 1, 4)
    gpu.mgq_update_sweeps(lat, beta, 3, 1, 1, 4)
    p_ref = orc.plaquette(U, dims)
    p_gpu = gpu.mgq_plaquette(lat)
    assert abs(p_gpu - p_ref) < 1e-6 * abs(p_ref), (p_gpu, p_ref)
    s_ref = orc.action(U, dims, beta)
    s_gpu = beta * 6 * U.shape[0] * (1 - p_gpu)
    assert abs(s_gpu - s_ref) < 1e-6 * abs(s_ref)
    assert gpu.mgq_check_unitarity(lat) < 5e-6


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32c12", 2e-5)])
def test_full_size_32x4_sampled_links(gpu, orc, prec, tol):
    """32^4 (the benchmark lattice, same launch configuration): one heat-bath
    sub-sweep on the GPU, sampled links recomputed one by one by the oracle."""
    dims, beta, seed = [32, 32, 32, 32], 6.0, 21
    U = orc.init_links(dims, 1, seed=seed)
    lat = _lat(gpu, dims, prec, seed=seed)
    lat.from_numpy(U)  # the FP32 lattice holds the rounded field; the oracle keeps FP64
    V = U.shape[0]
    dec = torch.full((V * 12,), 255, dtype=torch.uint8, device="cuda")
    gpu.mgq_heatbath_subsweep(lat, beta, 5, 1, 2, 1, dec)
    G = lat.to_numpy()
    d = dec.cpu().numpy().reshape(V, 4, 3)
    rng = np.random.default_rng(0)
    checked = 0
    while checked < 200:
        s = int(rng.integers(V))
        x = orc.coords(dims, s)
        if sum(x) % 2 != 1:
            continue
        ref, dref = orc.heatbath_one_link(U, dims, beta, seed, 0, 5, 1, s, 2)
        assert np.max(np.abs(G[s, 2] - ref)) < tol
        if prec == "f64":
            assert np.array_equal(d[s, 2], dref)
        checked += 1
    assert unitarity_violation(G[:, 2]) < (1e-13 if prec == "f64" else 2e-6)


def test_full_size_48x4_sampled_links(gpu, orc):
    """48^4 (the large-volume lattice, 5.3 M sites, the largest benchmarked
    extent; FP32 12-real): a heat-bath sub-sweep and then an overrelaxation
    sweep, sampled links recomputed by the oracle from the exact GPU input.
    The direction-0 even links of the overrelaxation sweep are updated first
    and never again, so they depend on the sweep's input field only."""
    dims, beta, seed = [48, 48, 48, 48], 6.2, 33
    lat = _lat(gpu, dims, "f32c12", seed=seed)
    gpu.mgq_init_links(lat, 1)
    U = lat.to_numpy()
    V = U.shape[0]
    gpu.mgq_heatbath_subsweep(lat, beta, 7, 1, 3, 0)
    G = lat.to_numpy()
    rng = np.random.default_rng(1)
    sites = rng.integers(V, size=4000)
    hb = [int(s) for s in sites if sum(orc.coords(dims, int(s))) % 2 == 0][:150]
    for s in hb:
        ref, _ = orc.heatbath_one_link(U, dims, beta, seed, 0, 7, 1, s, 3)
        assert np.max(np.abs(G[s, 3] - ref)) < 2e-5
    del U
    gpu.mgq_overrelax_sweep(lat)
    H = lat.to_numpy()
    for s in hb:  # even sites: direction 0 is the first sub-sweep
        ref = orc.overrelax_one_link(G, dims, s, 0)
        assert np.max(np.abs(H[s, 0] - ref)) < 2e-5
    assert unitarity_violation(H[:, 0]) < 2e-6


def test_plaquette_parity(gpu, orc):
    dims = [6, 4, 8, 2]
    U = orc.init_links(dims, 1, seed=3)
    orc.update_chain(U, dims, 5.7, 3, 0, 0, 3, 1, 1)
    for prec, tol in [("f64", 1e-14), ("f32", 1e-6), ("f32c12", 1e-6)]:
        lat = _lat(gpu, dims, prec)
        lat.from_numpy(U)
        assert abs(gpu.mgq_plaquette(lat) - orc.plaquette(U, dims)) < tol
    lat = _lat(gpu, dims)
    gpu.mgq_init_links(lat, 0)
    assert gpu.mgq_plaquette(lat) == 1.0


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32c12", 1e-6)])
@pytest.mark.parametrize("dims", [[6, 4, 4, 10], [8, 8, 8, 8]])
def test_overrelax_sweep_with_plaquette(gpu, orc, prec, tol, dims):
    """The overrelaxation sweep that measures the plaquette as it goes leaves
    the same links as the plain sweep, and its plaquette is the plaquette of
    those links (FP64: also the oracle's after its own sweep)."""
    U = orc.init_links(dims, 1, seed=44)
    orc.update_chain(U, dims, 5.8, 44, 0, 0, 3, 1, 1)
    a, b = _lat(gpu, dims, prec, seed=44), _lat(gpu, dims, prec, seed=44)
    a.from_numpy(U)
    b.from_numpy(U)
    orc.overrelax_sweep(U, dims)
    for k in range(2):  # twice in a row: the per-block sums start afresh
        p = gpu.mgq_overrelax_sweep_plaquette(a)
        gpu.mgq_overrelax_sweep(b)
        torch.cuda.synchronize()
        assert torch.equal(a.links, b.links)
        ref = gpu.mgq_plaquette(b)
        assert abs(p - ref) < tol * ref, (p, ref)
        if k == 0 and prec == "f64":
            assert abs(p - orc.plaquette(U, dims)) < 1e-12
    plaq = gpu.mgq_update_sweeps(b, 5.8, 9, 2, 1, 3, plaq_out=True)
    assert abs(plaq[-1] - gpu.mgq_plaquette(b)) < tol


def test_zero_sweeps_change_nothing(gpu):
    """Degenerate counts: no compound sweep leaves every link as it was, single
    and batched, with an empty plaquette record."""
    lats = [_lat(gpu, d, "f32c12", seed=11 + i, lid=i) for i, d in enumerate([[4, 4, 4, 4], [6, 4, 2, 8]])]
    for l in lats:
        gpu.mgq_init_links(l, 1)
    before = [l.links.clone() for l in lats]
    rec = gpu.mgq_update_sweeps(lats[0], 6.0, 0, 0, 1, 4, plaq_out=True)
    assert rec.size == 0
    B = gpu.Batch(lats, [6.0, 5.9])
    gpu.mgq_update_sweeps_batched(B, 0, 0, 1, 4)
    torch.cuda.synchronize()
    for l, b in zip(lats, before):
        assert torch.equal(l.links, b)


def test_heatbath_only_sweeps_parity(gpu, orc):
    """n_or = 0: compound sweeps of the heat bath alone, the plaquette then taken
    by the plaquette kernel (FP64: links 1e-12, plaquettes 1e-13)."""
    dims, beta = [4, 6, 4, 2], 5.8
    U = orc.init_links(dims, 1, seed=19)
    lat = _lat(gpu, dims, seed=19)
    lat.from_numpy(U)
    ref = orc.update_chain(U, dims, beta, 19, 0, 4, 2, 1, 0)
    got = gpu.mgq_update_sweeps(lat, beta, 4, 2, 1, 0, plaq_out=True)
    assert np.max(np.abs(got - ref)) < 1e-13
    assert np.max(np.abs(lat.to_numpy() - U)) < 1e-12
