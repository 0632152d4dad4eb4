"""GPU batched driver (independent lattices of uneven extents in one launch per
sub-sweep): bit-identical to separate single-lattice runs, per-lattice FP64
plaquettes, CUDA-graph capture."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SHAPES = [[4, 4, 4, 4], [6, 6, 6, 6], [4, 4, 4, 8], [8, 8, 8, 8], [2, 4, 6, 8]]


def _make(gpu, orc, prec, shapes, seed0=10):
    lats, singles, betas = [], [], []
    for i, d in enumerate(shapes):
        U = orc.init_links(d, 1, seed=seed0 + i, lattice_id=i)
        a = gpu.Lattice(d, prec, seed=seed0 + i, lattice_id=i)
        b = gpu.Lattice(d, prec, seed=seed0 + i, lattice_id=i)
        a.from_numpy(U)
        b.from_numpy(U)
        lats.append(a)
        singles.append(b)
        betas.append(5.8 + 0.3 * i / max(1, len(shapes) - 1))
    return lats, singles, betas


@pytest.mark.parametrize("prec", ["f64", "f32c12"])
def test_batched_equals_single_runs(gpu, orc, prec):
    lats, singles, betas = _make(gpu, orc, prec, SHAPES)
    batch = gpu.Batch(lats, betas, max_sweeps=4)
    P = batch.plaquette_buffer(3)
    gpu.mgq_update_sweeps_batched(batch, 7, 3, 1, 2, P)
    for i, (s, b) in enumerate(zip(singles, betas)):
        p = gpu.mgq_update_sweeps(s, b, 7, 3, 1, 2, plaq_out=True)
        assert np.array_equal(s.to_numpy(), lats[i].to_numpy()), i
        assert np.max(np.abs(P[:, i].cpu().numpy() - p)) < 1e-14, i


def test_batched_matches_oracle_fp64(gpu, orc):
    shapes = SHAPES[:3]
    lats, _, betas = _make(gpu, orc, "f64", shapes, seed0=30)
    batch = gpu.Batch(lats, betas, max_sweeps=2)
    P = batch.plaquette_buffer(1)
    gpu.mgq_update_sweeps_batched(batch, 0, 1, 1, 1, P)
    for i, d in enumerate(shapes):
        U = orc.init_links(d, 1, seed=30 + i, lattice_id=i)
        pref = orc.update_chain(U, d, betas[i], 30 + i, i, 0, 1, 1, 1)
        assert np.max(np.abs(lats[i].to_numpy() - U)) < 1e-11
        assert abs(P[0, i].item() - pref[0]) < 1e-12


def test_batched_graph_capture(gpu, orc):
    lats, singles, betas = _make(gpu, orc, "f32c12", SHAPES, seed0=50)
    batch = gpu.Batch(lats, betas, max_sweeps=2)
    P = batch.plaquette_buffer(1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        gpu.mgq_update_sweeps_batched(batch, 0, 1, 1, 1, P, stream=s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for i, b in enumerate(betas):
        gpu.mgq_update_sweeps(singles[i], b, 0, 1, 1, 1)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gpu.mgq_update_sweeps_batched(batch, 1, 1, 1, 1, P, stream=torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    for i, b in enumerate(betas):
        p = gpu.mgq_update_sweeps(singles[i], b, 1, 1, 1, 1, plaq_out=True)
        assert np.array_equal(singles[i].to_numpy(), lats[i].to_numpy()), i
        assert abs(P[0, i].item() - p[0]) < 1e-14


def test_batched_rejects_mixed_precision(gpu):
    a = gpu.Lattice([4, 4, 4, 4], "f64")
    b = gpu.Lattice([4, 4, 4, 4], "f32")
    with pytest.raises(gpu.MgqError):
        gpu.mgq_update_sweeps_batched(gpu.Batch([a, b], [6.0, 6.0]), 0, 1)
