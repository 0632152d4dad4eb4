"""mgq_plaquette_noalloc: the plaquette for callers that cannot hand the
library device memory (a framework that owns all device memory, or a hook
where cudaMalloc would synchronise the device).  It must agree with
mgq_plaquette, which reduces in the caller's workspace, on consecutive calls
through the C ABI; it keeps its scratch in a fixed static device array.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(lib, lat, out_ptr, stream):
    return lib.mgq_plaquette_noalloc(lat.ref, out_ptr, ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("dims,prec", [([8, 8, 8, 8], "f64"), ([6, 4, 2, 6], "f32"), ([32, 32, 32, 32], "f32c12")])
def test_noalloc_plaquette_matches_workspace_plaquette(gpu, mgqlib, dims, prec):
    stream = torch.cuda.current_stream()
    lat = gpu.Lattice(dims, prec, seed=5)
    gpu.mgq_init_links(lat, 1)
    gpu.mgq_update_sweeps(lat, 6.0, 0, 1, 1, 1)
    for call in range(2):  # two calls in a row share the static scratch
        ref = gpu.mgq_plaquette(lat)
        host = ctypes.c_double(-1.0)
        assert _noalloc(mgqlib, lat, ctypes.byref(host), stream) == 0, mgqlib.mgq_last_error()
        assert abs(host.value - ref) < 1e-14 * max(1.0, abs(ref)) + (1e-12 if prec != "f64" else 0.0), (call, host.value, ref)
        dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        assert _noalloc(mgqlib, lat, ctypes.c_void_p(dev.data_ptr()), stream) == 0
        assert abs(float(dev.item()) - ref) < 1e-14 * max(1.0, abs(ref)) + (1e-12 if prec != "f64" else 0.0)
        gpu.mgq_overrelax_sweep(lat)  # change the field between the two calls


def test_noalloc_rejects_lattices_beyond_its_scratch(gpu, mgqlib):
    from paper_1510_04675_gb300._lib import MgqLattice

    c = MgqLattice()
    c.dims[:] = [48, 48, 48, 48]   # 5.3M sites > the 2,096,896-site limit
    c.prec = 2
    c.links = 1 << 20   # never dereferenced: the size check comes first
    out = ctypes.c_double()
    assert mgqlib.mgq_plaquette_noalloc(ctypes.byref(c), ctypes.byref(out), None) == 1
    assert b"limit" in mgqlib.mgq_last_error()
