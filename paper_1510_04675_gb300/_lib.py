"""ctypes binding to libmgq.so: the mgq_lattice struct and every entry point
declared in include/mgq.h.  Loading fails loudly when the library has not
been built: there is no fallback path."""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmgq.so")

MGQ_OK, MGQ_EINVAL, MGQ_ENOMEM, MGQ_ECUDA, MGQ_EUNSUPPORTED, MGQ_ETIMEOUT, MGQ_ENONUNITARY = range(7)
MGQ_F64, MGQ_F32, MGQ_F32_C12 = 0, 1, 2
MGQ_WILSON = 0
MGQ_KERNEL_HEATBATH, MGQ_KERNEL_OVERRELAX = 0, 1
MGQ_PERIODIC, MGQ_OPEN = 0, 1


class MgqLattice(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int32 * 4),
        ("bc", ctypes.c_int32 * 4),
        ("prec", ctypes.c_int32),
        ("action", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("lattice_id", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("links", ctypes.c_void_p),
        ("mom", ctypes.c_void_p),
        ("work", ctypes.c_void_p),
        ("work_bytes", ctypes.c_uint64),
    ]


class MgqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mgq status {status}: {message}")
        self.status = status


_P = ctypes.POINTER(MgqLattice)
_vp, _d, _i, _u64, _u8p = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
_st = ctypes.c_int

# name -> (restype, argtypes); the status-returning calls are checked by call()
SIGNATURES = {
    "mgq_abi_version": (ctypes.c_int, []),
    "mgq_status_string": (ctypes.c_char_p, [_st]),
    "mgq_last_error": (ctypes.c_char_p, []),
    "mgq_site_stride": (ctypes.c_uint64, [ctypes.POINTER(ctypes.c_int32)]),
    "mgq_links_bytes": (ctypes.c_uint64, [_P]),
    "mgq_mom_bytes": (ctypes.c_uint64, [_P]),
    "mgq_workspace_bytes": (ctypes.c_uint64, [_P]),
    "mgq_init_links": (_st, [_P, _i, _vp]),
    "mgq_import_links": (_st, [_P, _vp, _vp]),
    "mgq_export_links": (_st, [_P, _vp, _vp]),
    "mgq_heatbath_sweep": (_st, [_P, _d, _u64, _i, _vp]),
    "mgq_heatbath_subsweep": (_st, [_P, _d, _u64, _i, _i, _i, _u8p, _vp]),
    "mgq_overrelax_sweep": (_st, [_P, _vp]),
    "mgq_overrelax_sweep_plaquette": (_st, [_P, _vp, _vp]),
    "mgq_update_sweeps": (_st, [_P, _d, _u64, _i, _i, _i, _vp, _vp]),
    "mgq_plaquette": (_st, [_P, _vp, _vp]),
    "mgq_plaquette_noalloc": (_st, [_P, _vp, _vp]),
    "mgq_topo_charge": (_st, [_P, _vp, _vp, _vp]),
    "mgq_topo_charge_improved": (_st, [_P, _vp, _vp]),
    "mgq_wilson_flow_times": (_st, [_P, _d, _d, _vp, _i, _i, _vp, _vp, _vp]),
    "mgq_wilson_loop": (_st, [_P, _i, _i, _vp, _vp]),
    "mgq_partial_loops": (_st, [_P, _vp, _vp]),
    "mgq_wilson_flow": (_st, [_P, _d, _i, _i, _vp, _vp, _vp]),
    "mgq_wilson_flow_adaptive": (_st, [_P, _d, _d, _d, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _u64, _vp]),
    "mgq_flow_adaptive_scratch_bytes": (ctypes.c_uint64, [_P]),
    "mgq_flow_adaptive_measurements": (ctypes.c_int, [_d, _d]),
    "mgq_hmc_force": (_st, [_P, _d, _vp, _vp]),
    "mgq_hmc_momentum_step": (_st, [_P, _d, _d, _vp]),
    "mgq_fma_probe": (ctypes.c_uint64, [_i, _vp, _vp]),
    "mgq_link_exp_update": (_st, [_P, _vp, _d, _vp]),
    "mgq_flow_adjoint_scratch_bytes": (ctypes.c_uint64, [_P]),
    "mgq_flow_vjp": (_st, [_P, _vp, _d, _vp, _vp]),
    "mgq_exp_vjp": (_st, [_P, _vp, _vp, _vp, _vp]),
    "mgq_wilson_flow_step_adjoint": (_st, [_P, _d, _vp, _vp, _u64, _vp]),
    "mgq_clover_vjp_scratch_bytes": (ctypes.c_uint64, [_P]),
    "mgq_clover_vjp": (_st, [_P, _i, _d, _vp, _vp, _u64, _vp]),
    "mgq_hmc_trajectory": (_st, [_P, _d, _d, _i, _u64, _i, _vp, _vp, _vp]),
    "mgq_prolongate": (_st, [_P, _P, _d, _d, _i, _vp, _vp, _vp]),
    "mgq_prolongate_batched_workspace_bytes": (ctypes.c_uint64, [_P, _i]),
    "mgq_prolongate_batched": (_st, [_P, _P, _i, _d, _d, _i, _i, _vp, _vp, _vp, _vp, _u64, _vp]),
    "mgq_restrict": (_st, [_P, _P, _vp]),
    "mgq_check_unitarity": (_st, [_P, _d, _vp, _vp]),
    "mgq_reunitarize": (_st, [_P, _i, _vp]),
    "mgq_batch_workspace_bytes": (ctypes.c_uint64, [_P, _i, _i]),
    "mgq_set_block_size": (_st, [_i, _i, _i]),
    "mgq_get_block_size": (ctypes.c_int, [_i, _i]),
    "mgq_update_sweeps_batched": (_st, [_P, _i, ctypes.POINTER(ctypes.c_double), _u64, _i, _i, _i, _vp, _vp, _u64,
                                        _vp]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libmgq.so (built in-tree by paper_1510_04675_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmgq.so not found at {LIB_PATH}; build it with paper_1510_04675_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def call(name: str, *args) -> int:
    """Call an mgq entry point and raise MgqError unless it returns MGQ_OK."""
    L = load()
    status = getattr(L, name)(*args)
    if status != MGQ_OK:
        raise MgqError(status, L.mgq_last_error().decode())
    return status
