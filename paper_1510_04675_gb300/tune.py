"""Autotuner for the launch shape of the checkerboard sub-sweep kernels.

For a lattice shape and storage format it times every candidate block size of
the heat-bath and overrelaxation kernels with CUDA events on a scratch copy of
the lattice, installs the fastest with mgq_set_block_size, and caches the
choice in a JSON file keyed by device name, extents and format, so later runs
apply it without timing.  Small lattices gain most: a 8^4 sub-sweep has only
2048 links, i.e. 16 blocks of 128 threads for 152 SMs.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

import torch

from . import _lib, api
from ._lib import MGQ_KERNEL_HEATBATH, MGQ_KERNEL_OVERRELAX, call

CANDIDATES = (32, 64, 96, 128)
_KERNELS = {"heatbath": MGQ_KERNEL_HEATBATH, "overrelax": MGQ_KERNEL_OVERRELAX}


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
    extents and format; returns {"heatbath": threads, "overrelax": threads}."""
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
        choice, timings = {}, {}
        for kernel in _KERNELS:
            best = None
            for bs in candidates:
                set_block_size(kernel, lat.prec, bs)
                if kernel == "heatbath":
                    ms = _time(lambda: api.mgq_heatbath_sweep(scratch, beta, 0, 1), reps)
                else:
                    ms = _time(lambda: api.mgq_overrelax_sweep(scratch), reps)
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
