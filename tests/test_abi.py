"""The C ABI: libmgq.so loads without a GPU, exports every entry point that
include/mgq.h declares, and rejects invalid arguments on the host before any
device work (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mgq_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(mgqlib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(mgqlib, n)]
    assert not missing, missing


def test_binding_covers_the_header(mgqlib):
    from paper_1510_04675_gb300 import _lib

    assert set(_declared()) <= set(_lib.SIGNATURES), set(_declared()) - set(_lib.SIGNATURES)


def _lat(dims=(4, 4, 4, 4), prec=0, bc=(0, 0, 0, 0)):
    from paper_1510_04675_gb300._lib import MgqLattice

    c = MgqLattice()
    c.dims[:] = list(dims)
    c.bc[:] = list(bc)
    c.prec = prec
    return c


def test_sizes(mgqlib):
    c = _lat((32, 32, 32, 32), 2)
    S = mgqlib.mgq_site_stride((ctypes.c_int32 * 4)(32, 32, 32, 32))
    assert S == 32**4 // 2
    assert mgqlib.mgq_links_bytes(ctypes.byref(c)) == 4 * 2 * 6 * S * 8
    assert mgqlib.mgq_mom_bytes(ctypes.byref(c)) == 4 * 2 * 8 * S * 4
    c = _lat((6, 6, 6, 6), 0)
    S = mgqlib.mgq_site_stride((ctypes.c_int32 * 4)(6, 6, 6, 6))
    assert S % 64 == 0 and S >= 648
    assert mgqlib.mgq_links_bytes(ctypes.byref(c)) == 4 * 2 * 9 * S * 16
    assert mgqlib.mgq_links_bytes(ctypes.byref(_lat((3, 4, 4, 4)))) == 0
    assert mgqlib.mgq_links_bytes(ctypes.byref(_lat((4, 4, 4, 4), 7))) == 0
    # the largest accepted volume is 2^28 sites (128^4); one more factor of two is refused
    assert mgqlib.mgq_links_bytes(ctypes.byref(_lat((128, 128, 128, 128), 2))) == 4 * 2 * 6 * 2**27 * 8
    assert mgqlib.mgq_links_bytes(ctypes.byref(_lat((256, 128, 128, 128), 2))) == 0
    assert mgqlib.mgq_site_stride((ctypes.c_int32 * 4)(128, 128, 128, 256)) == 0


@pytest.mark.parametrize("dims,prec,bc,status", [
    ((3, 4, 4, 4), 0, (0, 0, 0, 0), 1),   # odd extent
    ((0, 4, 4, 4), 0, (0, 0, 0, 0), 1),
    ((4, 4, 4, 4), 5, (0, 0, 0, 0), 1),   # bad precision
    ((4, 4, 4, 4), 0, (1, 0, 0, 0), 4),   # open boundary: unsupported
    ((4, 4, 4, 4), 0, (0, 0, 2, 0), 1),
    ((128, 256, 128, 128), 2, (0, 0, 0, 0), 1),  # volume 2^29 > 2^28
])
def test_host_side_rejections(mgqlib, dims, prec, bc, status):
    c = _lat(dims, prec, bc)
    c.links = 1 << 20  # never dereferenced: validation fails first
    assert mgqlib.mgq_heatbath_sweep(ctypes.byref(c), ctypes.c_double(5.7), ctypes.c_uint64(0), 1, None) == status
    assert mgqlib.mgq_last_error().decode()


def test_argument_ranges(mgqlib):
    c = _lat()
    c.links = 1 << 20
    f = mgqlib.mgq_heatbath_sweep
    assert f(ctypes.byref(c), ctypes.c_double(0.0), ctypes.c_uint64(0), 1, None) == 1      # beta <= 0
    assert f(ctypes.byref(c), ctypes.c_double(5.7), ctypes.c_uint64(0), 0, None) == 1      # n_hb < 1
    assert f(ctypes.byref(c), ctypes.c_double(5.7), ctypes.c_uint64(0), 257, None) == 1    # n_hb > 256
    assert mgqlib.mgq_heatbath_subsweep(ctypes.byref(c), ctypes.c_double(5.7), ctypes.c_uint64(0), 1, 4, 0,
                                        None, None) == 1
    c.links = None
    assert f(ctypes.byref(c), ctypes.c_double(5.7), ctypes.c_uint64(0), 1, None) == 1
    c.links = (1 << 20) + 8
    assert f(ctypes.byref(c), ctypes.c_double(5.7), ctypes.c_uint64(0), 1, None) == 1      # misaligned
    # workspace checks: missing / too small
    c.links = 1 << 20
    assert mgqlib.mgq_plaquette(ctypes.byref(c), ctypes.c_void_p(1 << 21), None) == 1
    c.work, c.work_bytes = 1 << 24, 1024
    assert mgqlib.mgq_plaquette(ctypes.byref(c), ctypes.c_void_p(1 << 21), None) == 2
    assert mgqlib.mgq_abi_version() == 1
    assert mgqlib.mgq_status_string(2) == b"workspace too small"


def test_block_size_settings(mgqlib):
    assert mgqlib.mgq_get_block_size(0, 2) == 128
    assert mgqlib.mgq_set_block_size(0, 2, 64) == 0 and mgqlib.mgq_get_block_size(0, 2) == 64
    assert mgqlib.mgq_set_block_size(0, 2, 128) == 0
    for bad in [(0, 2, 48), (0, 2, 256), (5, 0, 64), (-1, 0, 64), (1, 5, 64)]:
        assert mgqlib.mgq_set_block_size(*bad) == 1
    assert mgqlib.mgq_get_block_size(7, 0) == 0
    for k in range(5):  # single-lattice and batched sub-sweeps, APE
        assert mgqlib.mgq_get_block_size(k, 1) == 128


def test_adaptive_flow_host_helpers(mgqlib):
    from paper_1510_04675_gb300 import _lib

    f = _lib.load().mgq_flow_adaptive_measurements
    assert [f(1.0, 0.25), f(1.1, 0.25), f(0.0, 0.25), f(3.65, 0.1825)] == [5, 6, 1, 21]
    assert f(-1.0, 0.25) == -1 and f(1.0, 0.0) == -1 and f(float("nan"), 0.25) == -1
    c = _lat((8, 8, 8, 8), 2)
    assert _lib.load().mgq_flow_adaptive_scratch_bytes(ctypes.byref(c)) == 4 * 2 * 8 * 8**4 // 2 * 4


def test_empty_batches_are_refused(mgqlib):
    """A batch of no lattices is an argument error, refused before any work is queued."""
    c = _lat()
    c.links = 1 << 20
    betas = (ctypes.c_double * 1)(6.0)
    assert mgqlib.mgq_batch_workspace_bytes(ctypes.byref(c), 0, 1) == 0
    assert mgqlib.mgq_update_sweeps_batched(ctypes.byref(c), 0, betas, ctypes.c_uint64(0), 1, 1, 4, None, None,
                                            ctypes.c_uint64(0), None) == 1
    assert b"at least one" in mgqlib.mgq_last_error()
    f = _lat((8, 8, 8, 8))
    f.links = 1 << 20
    assert mgqlib.mgq_prolongate_batched_workspace_bytes(ctypes.byref(f), 0) == 0
    assert mgqlib.mgq_prolongate_batched(ctypes.byref(c), ctypes.byref(f), 0, ctypes.c_double(0.05),
                                         ctypes.c_double(1e-5), 100, 0, None, None, None, None,
                                         ctypes.c_uint64(0), None) == 1
    assert b"at least one" in mgqlib.mgq_last_error()
