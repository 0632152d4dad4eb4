"""The largest accepted lattice, 128^4 = 2^28 sites (FP32 12-real links,
51.5 GB, plus a 86 GB workspace): every 32-bit index the kernels form reaches
its maximum here.  A heat-bath sub-sweep (Sec. IV.A) from a cold start is
checked link by link on sampled links spread over the whole lattice, up to the
last sites: on a cold start every staple is 6 x identity, so the oracle's
lattice-free heat-bath map gives each updated link from its site index alone.
Then a full compound sweep runs, with properties that hold at any size."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

_EYE = np.eye(3, dtype=np.complex128)


def _sampled_links(lat, mu, sites):
    """Links U_mu(s) read straight from the paired 12-real device layout
    links[mu][parity][h/32][pair][h%32][4] (three 16-byte words per link:
    (u00, u01), (u02, u10), (u11, u12)); row 2 rebuilt as conj(row0 x row1)."""
    S = lat.site_stride
    L = lat.dims
    out = []
    f = lat.links.view(torch.float32)
    idx = []
    for s in sites:
        x = [s % L[0], (s // L[0]) % L[1], (s // (L[0] * L[1])) % L[2], s // (L[0] * L[1] * L[2])]
        par, h = sum(x) & 1, s >> 1
        block = (mu * 2 + par) * (S >> 5) + (h >> 5)
        base = block * 96 + (h & 31)
        for k in range(3):
            idx.extend(4 * (base + 32 * k) + np.arange(4))
    vals = f[torch.tensor(idx, dtype=torch.int64, device=f.device)].double().cpu().numpy().reshape(len(sites), 12)
    for v in vals:
        c = v[0::2] + 1j * v[1::2]  # u00 u01 u02 u10 u11 u12
        U = np.zeros((3, 3), dtype=np.complex128)
        U[0], U[1] = c[:3], c[3:]
        U[2] = np.conj(np.cross(U[0], U[1]))
        out.append(U)
    return out


def test_layout_reader_matches_export(gpu):
    """The layout reader above against the library's own export (ragged 6x4x4x10:
    a partly filled last 32-site block)."""
    dims = [6, 4, 4, 10]
    lat = gpu.Lattice(dims, "f32c12", seed=5)
    gpu.mgq_init_links(lat, 1)
    U = lat.to_numpy()
    sites = list(range(0, U.shape[0], 7)) + [U.shape[0] - 1]
    for mu in range(4):
        got = _sampled_links(lat, mu, sites)
        for s, g in zip(sites, got):
            assert np.max(np.abs(g - U[s, mu])) < 1e-6


def test_max_volume_128x4(gpu, orc):
    dims, beta, seed, lid, sweep, mu, par = [128, 128, 128, 128], 6.0, 41, 3, 9, 3, 1
    V = 2**28
    need = 137 * 2**30
    torch.cuda.empty_cache()
    if torch.cuda.mem_get_info()[0] < need:
        pytest.skip("needs about 140 GB of free device memory")
    lat = gpu.Lattice(dims, "f32c12", seed=seed, lattice_id=lid)
    try:
        gpu.mgq_init_links(lat, 0)
        gpu.mgq_heatbath_subsweep(lat, beta, sweep, 1, mu, par)
        torch.cuda.synchronize()
        rng = np.random.default_rng(7)
        cand = [V - 2, V - 4, V - 2**20 - 1, 2**27 - 1, 2**27 + 1, 1] + [int(s) for s in rng.integers(V, size=600)]
        upd = [s for s in cand if (sum(orc.coords(dims, s)) & 1) == par][:260]
        assert V - 2 in upd and 2**27 + 1 in upd  # the last sites of the lattice are checked
        for s, G in zip(upd, _sampled_links(lat, mu, upd)):
            ref, _ = orc.heatbath_link_staple(_EYE, 6 * _EYE, beta, seed, lid, sweep, 1, s, mu)
            assert np.max(np.abs(G - ref)) < 2e-5, s
        # links outside the (mu, parity) subset are untouched
        other = [s for s in cand if (sum(orc.coords(dims, s)) & 1) != par][:64]
        for m, sites in ((mu, other), (0, upd[:64]), (2, other)):
            for G in _sampled_links(lat, m, sites):
                assert np.array_equal(G, _EYE)
        # a full compound sweep (1 HB + 4 OR) with the folded plaquette
        plaq = gpu.mgq_update_sweeps(lat, beta, sweep + 1, 1, 1, 4, plaq_out=True)
        assert np.all(np.isfinite(plaq)) and 0.0 < plaq[-1] < 1.0
        assert abs(plaq[-1] - gpu.mgq_plaquette(lat)) < 1e-6  # FP32 products, two summation orders
        assert gpu.mgq_check_unitarity(lat) < 2e-6
        last = _sampled_links(lat, 3, [V - 1, V - 2])
        assert all(np.max(np.abs(G - _EYE)) > 1e-3 for G in last)  # the last links were updated
    finally:
        del lat
        torch.cuda.empty_cache()
