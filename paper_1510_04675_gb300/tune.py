"""Autotuner for the launch shapes of the tunable kernels.

For a lattice (or a batch of lattices, or a prolongation batch) it times every
candidate block size of the heat-bath and overrelaxation sub-sweep kernels --
single-lattice and batched -- and of the APE step of the prolongation with
CUDA events, installs the fastest with mgq_set_block_size, and caches the
choice in a JSON file keyed by device name, kernel family, extents and format,
so later runs apply it without timing.  Small lattices gain most: a 8^4
sub-sweep has only 2048 links, i.e. 16 blocks of 128 threads for 152 SMs.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

import torch

from . import _lib, api
from ._lib import MGQ_KERNEL_HEATBATH, MGQ_KERNEL_OVERRELAX, call

CANDIDATES = (32, 64, 96, 128)
STAGED_THREADS = 128  # block size of the staged FP32 12-real sub-sweeps (not tunable)
STAGED_MIN_VH = 49152  # single-lattice FP32 12-real sub-sweeps are staged from V/2 >= this on
_KERNELS = {"heatbath": MGQ_KERNEL_HEATBATH, "overrelax": MGQ_KERNEL_OVERRELAX, "heatbath_batched": 2,
            "overrelax_batched": 3, "ape": 4}


def default_cache_path() -> str:
    return os.environ.get("MGQ_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "mgq", "tune.json"))


def _key(lat: "api.Lattice") -> str:
    name = torch.cuda.get_device_name(lat.device)
    return f"{name}|{'x'.join(map(str, lat.dims))}|{lat.prec}"


def set_block_size(kernel: str, prec: str, threads: int) -> None:
    call("mgq_set_block_size", _KERNELS[kernel], api.PRECISIONS[prec], int(threads))


def get_block_size(kernel: str, prec: str) -> int:
    return int(_lib.load().mgq_get_block_size(_KERNELS[kernel], api.PRECISIONS[prec]))


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def autotune(lat: "api.Lattice", beta: float = 6.0, candidates: Sequence[int] = CANDIDATES, reps: int = 5,
             cache_path: Optional[str] = None, use_cache: bool = True) -> Dict[str, int]:
    """Choose and install the fastest block size per kernel for this lattice's
    extents and format; returns {"heatbath": threads, "overrelax": threads}.
    FP32 12-real sub-sweeps of lattices with V/2 >= STAGED_MIN_VH stage their
    staple links through shared memory at a fixed 128 threads per block; for
    them the candidates time alike and the choice has no effect."""
    path = cache_path or default_cache_path()
    key = _key(lat)
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        choice = cache[key]
    else:
        scratch = api.copy_lattice(lat)
        plaq = torch.zeros(1, dtype=torch.float64, device=lat.device)
        choice, timings = {}, {}
        for kernel in ("heatbath", "overrelax"):
            best = None
            for bs in candidates:
                set_block_size(kernel, lat.prec, bs)
                if kernel == "heatbath":
                    ms = _time(lambda: api.mgq_heatbath_sweep(scratch, beta, 0, 1), reps)
                else:
                    # the overrelaxation sweeps of a compound sweep: plain ones and the
                    # last one, which measures the plaquette with the same block size
                    ms = _time(lambda: [api.mgq_overrelax_sweep(scratch) for _ in range(3)]
                               + [api.mgq_overrelax_sweep_plaquette(scratch, out=plaq)], reps)
                timings[f"{kernel}:{bs}"] = ms
                if best is None or ms < best[1]:
                    best = (bs, ms)
            choice[kernel] = best[0]
        cache[key] = choice
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    for kernel, bs in choice.items():
        set_block_size(kernel, lat.prec, bs)
    return dict(choice)


def _cached(key: str, cache_path: Optional[str], use_cache: bool, measure) -> Dict[str, int]:
    path = cache_path or default_cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        return dict(cache[key])
    choice = measure()
    cache[key] = choice
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    return choice


def autotune_batched(batch: "api.Batch", candidates: Sequence[int] = CANDIDATES, reps: int = 3,
                     cache_path: Optional[str] = None, use_cache: bool = True) -> Dict[str, int]:
    """Block sizes of the batched heat-bath and overrelaxation kernels for this
    batch's lattice shapes: the heat bath timed alone (sweeps without
    overrelaxation), then the overrelaxation inside compound sweeps (1 HB + 4 OR)
    with the chosen heat-bath size.  The batch's links are advanced by the timing."""
    prec = batch.lattices[0].prec
    if prec == "f32c12":  # staged sub-sweeps, a fixed 128 threads per block
        return {"heatbath_batched": STAGED_THREADS, "overrelax_batched": STAGED_THREADS}
    shapes = sorted({"x".join(map(str, l.dims)) for l in batch.lattices})
    key = f"{torch.cuda.get_device_name(batch.lattices[0].device)}|batched|{batch.n}|{','.join(shapes)}|{prec}"

    def measure():
        choice = {}
        for kernel, n_or in (("heatbath_batched", 0), ("overrelax_batched", 4)):
            best = None
            for bs in candidates:
                set_block_size(kernel, prec, bs)
                ms = _time(lambda: api.mgq_update_sweeps_batched(batch, 0, 1, 1, n_or), reps)
                if best is None or ms < best[1]:
                    best = (bs, ms)
            choice[kernel] = best[0]
            set_block_size(kernel, prec, best[0])
        return choice

    choice = _cached(key, cache_path, use_cache, measure)
    for kernel, bs in choice.items():
        set_block_size(kernel, prec, bs)
    return dict(choice)


def autotune_ape(pbatch: "api.ProlongBatch", candidates: Sequence[int] = CANDIDATES, iterations: int = 24,
                 reps: int = 2, cache_path: Optional[str] = None, use_cache: bool = True) -> Dict[str, int]:
    """Block size of the APE step of the prolongation for this batch's fine
    shapes, timed on a fixed budget of `iterations` APE iterations (the fine
    lattices are overwritten)."""
    prec = pbatch.fine[0].prec
    shapes = sorted({"x".join(map(str, l.dims)) for l in pbatch.fine})
    key = f"{torch.cuda.get_device_name(pbatch.fine[0].device)}|ape|{pbatch.n}|{','.join(shapes)}|{prec}"

    def measure():
        best = None
        for bs in candidates:
            set_block_size("ape", prec, bs)
            ms = _time(lambda: api.mgq_prolongate_batched(pbatch, 0.05, 0.0, 10000, iter_budget=iterations), reps)
            if best is None or ms < best[1]:
                best = (bs, ms)
        return {"ape": best[0]}

    choice = _cached(key, cache_path, use_cache, measure)
    set_block_size("ape", prec, choice["ape"])
    return dict(choice)

