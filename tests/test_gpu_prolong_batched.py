"""Device-side stopping rule and batched prolongation (Sec. III, Eqs.
prolongation, smoothing, APE; Sec. IV.C's 0.001 % rule; Sec. II: many
configurations refined in parallel), and two refinement levels against the
FP64 oracle."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _coarse(orc, dims, beta=5.7, seed=1, n=4):
    U = orc.init_links(dims, 1, seed=seed)
    orc.update_chain(U, dims, beta, seed, 0, 0, n, 1, 2)
    return U


def test_batched_prolongation_matches_oracle_fp64(gpu, orc):
    shapes = [[2, 2, 2, 4], [2, 4, 2, 2], [4, 2, 4, 2]]   # uneven extents in one call
    coarse, fine, refs = [], [], []
    for i, dc in enumerate(shapes):
        Uc = _coarse(orc, dc, seed=10 + i)
        refs.append(orc.prolongate(Uc, dc, 0.05, 1e-5, 5000))
        c = gpu.Lattice(dc, "f64")
        c.from_numpy(Uc)
        coarse.append(c)
        fine.append(gpu.Lattice([2 * v for v in dc], "f64"))
    B = gpu.ProlongBatch(coarse, fine)
    gpu.mgq_prolongate_batched(B, 0.05, 1e-5, 5000)
    iters, sd = B.iters.cpu().numpy(), B.sd.cpu().numpy()
    assert int(B.n_done.item()) == 3
    for i, (ref, it_ref, sd_ref) in enumerate(refs):
        assert list(iters[i]) == it_ref, (i, iters[i], it_ref)
        assert np.max(np.abs(sd[i] - sd_ref)) < 1e-9 * max(1.0, np.max(np.abs(sd_ref)))
        assert np.max(np.abs(fine[i].to_numpy() - ref)) < 1e-9


def _fp32_pairs(gpu, shapes, seed):
    coarse, fine = [], []
    for i, dc in enumerate(shapes):
        c = gpu.Lattice(dc, "f32c12", seed=seed + i)
        gpu.mgq_init_links(c, 1)
        gpu.mgq_update_sweeps(c, 5.8, 0, 10, 1, 2)
        coarse.append(c)
        fine.append(gpu.Lattice([2 * v for v in dc], "f32c12"))
    return coarse, fine


def test_batched_equals_single_lattice_calls(gpu):
    shapes = [[8, 8, 8, 8], [6, 6, 6, 6], [4, 4, 4, 8]]
    coarse, fine = _fp32_pairs(gpu, shapes, 40)
    B = gpu.ProlongBatch(coarse, fine)
    gpu.mgq_prolongate_batched(B, 0.05, 1e-5, 10000)
    for i, c in enumerate(coarse):
        f1 = gpu.Lattice(fine[i].dims, "f32c12")
        iters, sd = gpu.mgq_prolongate(c, f1, 0.05, 1e-5, 10000)
        assert list(B.iters[i].cpu().numpy()) == iters
        assert np.array_equal(B.sd[i].cpu().numpy(), np.array(sd))
        assert torch.equal(f1.links, fine[i].links)


def test_iteration_budget_in_a_cuda_graph(gpu):
    shapes = [[8, 8, 8, 8], [6, 6, 6, 6]]
    coarse, fine = _fp32_pairs(gpu, shapes, 50)
    B = gpu.ProlongBatch(coarse, fine)
    gpu.mgq_prolongate_batched(B, 0.05, 1e-5, 10000)        # run to completion
    need = int(B.iters.sum(dim=1).max().item()) + 3
    ref_links = [f.links.clone() for f in fine]
    ref_iters = B.iters.clone()
    for f in fine:
        f.links.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):   # warm up the code path outside the capture
        gpu.mgq_prolongate_batched(B, 0.05, 1e-5, 10000, iter_budget=need, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gpu.mgq_prolongate_batched(B, 0.05, 1e-5, 10000, iter_budget=need + 7,
                                   stream=torch.cuda.current_stream())
    for f in fine:
        f.links.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert int(B.n_done.item()) == 2
    assert torch.equal(B.iters, ref_iters)
    for f, r in zip(fine, ref_links):
        assert torch.equal(f.links, r)
    # too small a budget: the lattices are not finished and say so
    gpu.mgq_prolongate_batched(B, 0.05, 1e-5, 10000, iter_budget=need // 2)
    torch.cuda.synchronize()
    assert int(B.n_done.item()) == 0
    assert int(B.iters[:, 2].sum().item()) == 0


def test_two_level_refinement_matches_oracle_fp64(gpu, orc):
    """Coarsest 2x2x2x4 -> 4x4x4x8 -> 8x8x8x16 with one heat-bath sweep of the
    middle level in between (Sec. I-II: several refinement levels)."""
    d0, beta, seed, lid = [2, 2, 2, 4], 6.0, 77, 5
    d1, d2 = [2 * v for v in d0], [4 * v for v in d0]
    U0 = _coarse(orc, d0, seed=21)
    U1, it1, _ = orc.prolongate(U0, d0, 0.05, 1e-5, 5000)
    dref = orc.new_decisions(d1)
    orc.heatbath_sweep(U1, d1, beta, seed, lid, 3, 1, dref)
    U2, it2, _ = orc.prolongate(U1, d1, 0.05, 1e-5, 5000)

    l0 = gpu.Lattice(d0, "f64")
    l0.from_numpy(U0)
    l1 = gpu.Lattice(d1, "f64", seed=seed, lattice_id=lid)
    l2 = gpu.Lattice(d2, "f64")
    g1, _ = gpu.mgq_prolongate(l0, l1, 0.05, 1e-5, 5000)
    V1 = U1.shape[0]
    dgpu = torch.full((V1 * 12,), 255, dtype=torch.uint8, device="cuda")
    for mu in range(4):
        for par in range(2):
            gpu.mgq_heatbath_subsweep(l1, beta, 3, 1, mu, par, dgpu)
    assert np.array_equal(dgpu.cpu().numpy().reshape(V1, 4, 3), dref)
    assert np.max(np.abs(l1.to_numpy() - U1)) < 1e-9
    g2, _ = gpu.mgq_prolongate(l1, l2, 0.05, 1e-5, 5000)
    assert g1 == it1 and g2 == it2, (g1, it1, g2, it2)
    assert np.max(np.abs(l2.to_numpy() - U2)) < 1e-8
