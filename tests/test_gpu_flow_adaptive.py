"""GPU adaptive-step Wilson flow (Sec. IV.B, Table II) against the oracle:
FP64 step-by-step parity (same accepted/rejected trials, same E, Q and
links), FP32 formats, the loose-tolerance limit (the fixed-step flow), the
underflow error, and the paper's fixed-vs-adaptive deviation at full size."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _thermal(orc, dims, beta, seed, n):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 4)
    return U


def test_adaptive_parity_fp64(gpu, orc):
    """Ragged 6x4x4x10 lattice, oversized first trial (rejections), t_end not a
    multiple of dt_meas: identical step/reject counts, E, Q and links."""
    dims = [6, 4, 4, 10]
    U = _thermal(orc, dims, 5.626, 21, 20)
    W = U.copy()
    E_ref, Q_ref, s_ref, r_ref = orc.wilson_flow_adaptive(W, dims, 1.1, 1e-3, 0.2, 0.2, 0.25)
    lat = gpu.Lattice(dims, "f64")
    lat.from_numpy(U)
    E, Q, s, r = gpu.mgq_wilson_flow_adaptive(lat, 1.1, 1e-3, 0.2, 0.2, 0.25)
    assert r_ref >= 1 and (s, r) == (s_ref, r_ref)
    assert len(E) == len(E_ref) == 6
    assert np.max(np.abs(E - E_ref) / E_ref) < 1e-10 and np.max(np.abs(Q - Q_ref)) < 1e-10
    assert np.max(np.abs(lat.to_numpy() - W)) < 1e-10


@pytest.mark.parametrize("prec", ["f32", "f32c12"])
def test_adaptive_fp32_formats(gpu, orc, prec):
    dims = [8, 8, 8, 8]
    U = _thermal(orc, dims, 5.626, 22, 20)
    E_ref, Q_ref, s_ref, r_ref = orc.wilson_flow_adaptive(U.copy(), dims, 1.8, 1e-4, 0.2, 0.01, 0.18)
    lat = gpu.Lattice(dims, prec)
    lat.from_numpy(U)
    E, Q, s, r = gpu.mgq_wilson_flow_adaptive(lat, 1.8, 1e-4, 0.2, 0.01, 0.18)
    assert len(E) == len(E_ref) == 11
    assert abs(s - s_ref) <= 1 and abs(r - r_ref) <= 1, (s, s_ref, r, r_ref)
    assert np.max(np.abs(E - E_ref) / E_ref) < 3e-5, (E, E_ref)
    assert np.max(np.abs(Q - Q_ref)) < 2e-3


def test_adaptive_loose_tolerance_is_fixed_step_flow(gpu, orc):
    dims = [4, 6, 4, 4]
    U = _thermal(orc, dims, 6.0, 23, 5)
    a, b = gpu.Lattice(dims, "f64"), gpu.Lattice(dims, "f64")
    a.from_numpy(U)
    b.from_numpy(U)
    E, Q, s, r = gpu.mgq_wilson_flow_adaptive(a, 1.0, 1e9, 0.0625, 0.0625, 0.25)
    Ef, Qf = gpu.mgq_wilson_flow(b, 0.0625, 16, 4)
    assert (s, r) == (16, 0)
    assert np.max(np.abs(E - Ef)) < 1e-12 and np.max(np.abs(Q - Qf)) < 1e-12
    assert np.max(np.abs(a.to_numpy() - b.to_numpy())) < 1e-13


def test_adaptive_step_underflow_is_reported(gpu, orc):
    """A tolerance below FP32 rounding can never be met: the controller stops
    with an error and the links are those at the last kept step (here the
    start)."""
    dims = [4, 4, 4, 4]
    U = _thermal(orc, dims, 5.7, 24, 5)
    lat = gpu.Lattice(dims, "f32c12")
    lat.from_numpy(U)
    before = lat.to_numpy()
    with pytest.raises(gpu.MgqError, match="underflow"):
        gpu.mgq_wilson_flow_adaptive(lat, 1.0, 1e-14, 0.2, 0.1, 0.25)
    assert np.array_equal(lat.to_numpy(), before)
    assert np.isfinite(gpu.mgq_plaquette(lat))


def test_adaptive_matches_fixed_flow_at_full_size(gpu):
    """Sec. IV.B on the 12^3 x 24, beta = 5.626 ensemble (t0 ~ 0.73):
    tolerance 0.01, maximal step 0.2, measurements every 0.18 ~ t0/4 up to
    3.6 ~ 5 t0.  E(t) deviates from the fixed-step (0.01) flow by less than
    the paper's 0.02 %, Q agrees per configuration, and the adaptive flow
    needs far fewer steps."""
    dims = [12, 12, 12, 24]
    for seed in (31, 32):
        lat = gpu.Lattice(dims, "f32c12", seed=seed)
        gpu.mgq_init_links(lat, 1)
        gpu.mgq_update_sweeps(lat, 5.626, 0, 200, 1, 4)
        ref = gpu.Lattice(dims, "f32c12")
        ref.from_numpy(lat.to_numpy())
        Ef, Qf = gpu.mgq_wilson_flow(ref, 0.01, 360, 18)
        E, Q, s, r = gpu.mgq_wilson_flow_adaptive(lat, 3.6, 0.01, 0.2, 0.01, 0.18)
        assert len(E) == len(Ef) == 21
        assert np.max(np.abs(E - Ef) / Ef) < 2e-4, np.abs(E - Ef) / Ef
        assert np.max(np.abs(Q - Qf)) < 0.01, (Q, Qf)
        assert s < 360 // 4, s
