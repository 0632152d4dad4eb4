"""Autotuner: picks one of the candidate block sizes, caches it, and the
results of a sweep do not depend on the launch shape (bit for bit)."""
import json

import pytest
import torch

pytestmark = pytest.mark.gpu


def test_autotune_and_launch_shape_independence(gpu, tmp_path):
    from paper_1510_04675_gb300 import tune

    lat = gpu.Lattice([8, 8, 8, 8], "f32c12", seed=4)
    gpu.mgq_init_links(lat, 1)
    cache = str(tmp_path / "tune.json")
    choice = tune.autotune(lat, cache_path=cache)
    assert set(choice) == {"heatbath", "overrelax"}
    assert all(v in tune.CANDIDATES for v in choice.values())
    assert json.load(open(cache))
    assert tune.autotune(lat, cache_path=cache) == choice          # served from the cache
    results = []
    for bs in (32, 128):
        tune.set_block_size("heatbath", "f32c12", bs)
        tune.set_block_size("overrelax", "f32c12", bs)
        c = gpu.copy_lattice(lat)
        gpu.mgq_update_sweeps(c, 6.0, 0, 2, 1, 2)
        results.append(c.links.clone())
    assert torch.equal(results[0], results[1])
    tune.set_block_size("heatbath", "f32c12", 128)
    tune.set_block_size("overrelax", "f32c12", 128)
