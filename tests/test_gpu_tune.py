"""Autotuner: picks one of the candidate block sizes, caches it, and the
results of a sweep do not depend on the launch shape (bit for bit)."""
import json

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_autotune_and_launch_shape_independence(gpu, tmp_path):
    from paper_1510_04675_gb300 import tune

    lat = gpu.Lattice([8, 8, 8, 8], "f32", seed=4)
    gpu.mgq_init_links(lat, 1)
    cache = str(tmp_path / "tune.json")
    choice = tune.autotune(lat, cache_path=cache)
    assert set(choice) == {"heatbath", "overrelax"}
    assert all(v in tune.CANDIDATES for v in choice.values())
    assert json.load(open(cache))
    assert tune.autotune(lat, cache_path=cache) == choice          # served from the cache
    results = []
    for bs in (32, 128):
        tune.set_block_size("heatbath", "f32", bs)
        tune.set_block_size("overrelax", "f32", bs)
        c = gpu.copy_lattice(lat)
        gpu.mgq_update_sweeps(c, 6.0, 0, 2, 1, 2)
        results.append(c.links.clone())
    assert torch.equal(results[0], results[1])
    tune.set_block_size("heatbath", "f32", 128)
    tune.set_block_size("overrelax", "f32", 128)


def test_batched_and_ape_shapes_tuned_and_result_independent(gpu, tmp_path):
    from paper_1510_04675_gb300 import tune

    shapes = [[8, 8, 8, 8], [6, 6, 6, 6], [4, 4, 4, 8]]
    lats = []
    for i, s in enumerate(shapes):
        l = gpu.Lattice(s, "f32", seed=7, lattice_id=i)
        gpu.mgq_init_links(l, 1)
        lats.append(l)
    cache = str(tmp_path / "tune.json")
    b = gpu.Batch([gpu.copy_lattice(l) for l in lats], [5.9] * 3)
    choice = tune.autotune_batched(b, cache_path=cache)
    assert set(choice) == {"heatbath_batched", "overrelax_batched"}
    fine = [gpu.Lattice([2 * v for v in s], "f32") for s in shapes]
    pb = gpu.ProlongBatch(lats, fine)
    ape = tune.autotune_ape(pb, cache_path=cache)
    assert ape["ape"] in tune.CANDIDATES
    sweeps, prol = [], []
    for bs in (32, 96):
        for k in ("heatbath_batched", "overrelax_batched", "ape"):
            tune.set_block_size(k, "f32", bs)
        c = [gpu.copy_lattice(l) for l in lats]
        gpu.mgq_update_sweeps_batched(gpu.Batch(c, [5.9] * 3), 0, 2, 1, 2)
        sweeps.append(torch.cat([x.links for x in c]))
        gpu.mgq_prolongate_batched(pb, 0.05, 1e-5, 10000)
        prol.append((torch.cat([f.links for f in fine]), pb.iters.clone()))
    assert torch.equal(sweeps[0], sweeps[1])
    assert torch.equal(prol[0][0], prol[1][0]) and torch.equal(prol[0][1], prol[1][1])
    for k in ("heatbath_batched", "overrelax_batched", "ape"):
        tune.set_block_size(k, "f32", 128)
