"""FP64 CPU oracle for the multiscale SU(3) thermalization hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package; the
product library (``paper_1510_04675_gb300``) never does.  The oracle shares
no code with the CUDA library.  It is a ctypes binding to ``mgq_oracle.c``
plus numpy conveniences.

Canonical layout of a gauge field: complex128 array of shape (V, 4, 3, 3),
site index ``x0 + L0*(x1 + L1*(x2 + L2*x3))`` (x0 fastest), then mu, row,
column.  Lie-algebra fields (momenta, forces): float64 (V, 4, 8),
coefficients of X_a = i lambda_a / 2.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mgq_oracle.c")
_SO = os.path.join(_HERE, "libmgq_oracle.so")

KIND_HB, KIND_HOT, KIND_MOM, KIND_ACCEPT = 1, 2, 3, 4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fcx-limited-range",
               "-fPIC", "-shared", "-o", _SO + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_u64, _u32, _int, _dbl, _long = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double, ctypes.c_long

_SIGS = {
    "orc_philox4x32_10": (None, [_U32, _U32, _U32]),
    "orc_draw_uniforms": (None, [_u64, _u32, _u32, _int, _int, _int, _int, _u64, _D]),
    "orc_plaquette": (_dbl, [_D, _I]),
    "orc_action": (_dbl, [_D, _I, _dbl]),
    "orc_staple": (None, [_D, _I, _long, _int, _D]),
    "orc_init_links": (None, [_D, _I, _int, _u64, _u32]),
    "orc_creutz_samples": (None, [_dbl, _u64, _long, _D, _I]),
    "orc_or_link_ordered": (None, [_D, _D, _I, _D]),
    "orc_heatbath_sweep": (None, [_D, _I, _dbl, _u64, _u32, _u64, _int, _U8]),
    "orc_heatbath_subsweep": (None, [_D, _I, _dbl, _u64, _u32, _u64, _int, _int, _int, _U8]),
    "orc_heatbath_one_link": (None, [_D, _I, _dbl, _u64, _u32, _u64, _int, _long, _int, _D, _U8]),
    "orc_heatbath_link_staple": (None, [_D, _D, _dbl, _u64, _u32, _u64, _int, _long, _int, _D, _U8]),
    "orc_overrelax_sweep": (None, [_D, _I]),
    "orc_overrelax_one_link": (None, [_D, _I, _long, _int, _D]),
    "orc_overrelax_subsweep": (None, [_D, _I, _int, _int]),
    "orc_subsweep_range": (None, [_D, _I, _int, _dbl, _u64, _u32, _u64, _int, _int, _int, _long, _long]),
    "orc_update_chain": (None, [_D, _I, _dbl, _u64, _u32, _u64, _int, _int, _int, _D]),
    "orc_expm": (None, [_D, _D]),
    "orc_alg_to_mat": (None, [_D, _D]),
    "orc_mat_to_alg": (None, [_D, _D]),
    "orc_force": (None, [_D, _I, _dbl, _D]),
    "orc_mom_refresh": (None, [_D, _I, _u64, _u32, _u64]),
    "orc_kinetic": (_dbl, [_D, _I]),
    "orc_update_links": (None, [_D, _D, _I, _dbl]),
    "orc_leapfrog": (None, [_D, _D, _I, _dbl, _dbl, _int]),
    "orc_hmc_trajectory": (None, [_D, _D, _I, _dbl, _dbl, _int, _u64, _u32, _u64, _int, _D, _I]),
    "orc_su3_project": (None, [_D, _int, _D]),
    "orc_reunit": (None, [_D, _D]),
    "orc_restrict": (None, [_D, _I, _D]),
    "orc_transfer": (None, [_D, _I, _D]),
    "orc_partial_action": (_dbl, [_D, _I, _int]),
    "orc_prolongate": (None, [_D, _I, _D, _dbl, _dbl, _int, _int, _I, _D]),
    "orc_ape_step": (None, [_D, _I, _int, _dbl, _int]),
    "orc_flow_step": (None, [_D, _I, _dbl]),
    "orc_wilson_loop": (_dbl, [_D, _I, _int, _int]),
    "orc_partial_loops": (None, [_D, _I, _D]),
    "orc_clover_EQ": (None, [_D, _I, _D, _D]),
    "orc_clover_q_site": (_dbl, [_D, _I, _long, _int]),
    "orc_topo_charge_improved": (None, [_D, _I, _D]),
    "orc_wilson_flow_times": (None, [_D, _I, _dbl, _dbl, _D, _int, _int, _D, _D]),
    "orc_wilson_flow": (None, [_D, _I, _dbl, _int, _int, _D, _D]),
    "orc_flow_trial_step": (_dbl, [_D, _I, _dbl]),
    "orc_wilson_flow_adaptive": (_int, [_D, _I, _dbl, _dbl, _dbl, _dbl, _dbl, _D, _D, _int, _I, _I]),
    "orc_set_threads": (None, [_int]),
    "orc_get_threads": (_int, []),
}


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ---------------------------------------------------------------- helpers
def _dims(dims) -> ctypes.Array:
    d = [int(v) for v in dims]
    assert len(d) == 4
    return (ctypes.c_int * 4)(*d)


def volume(dims) -> int:
    return int(np.prod([int(v) for v in dims]))


def _dp(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def new_field(dims) -> np.ndarray:
    return np.zeros((volume(dims), 4, 3, 3), dtype=np.complex128)


def site_index(dims, x) -> int:
    L = [int(v) for v in dims]
    s = 0
    for mu in (3, 2, 1, 0):
        s = s * L[mu] + (int(x[mu]) % L[mu])
    return s


def coords(dims, s: int):
    L = [int(v) for v in dims]
    x = []
    for mu in range(4):
        x.append(s % L[mu])
        s //= L[mu]
    return x


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# ---------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def draw_uniforms(seed, lattice_id, site, mu, subgroup, attempt, kind, sweep):
    u = np.zeros(4)
    lib().orc_draw_uniforms(seed, lattice_id, site, mu, subgroup, attempt, kind, sweep, _dp(u))
    return u


# ---------------------------------------------------------------- fields
def init_links(dims, start: int, seed: int = 0, lattice_id: int = 0) -> np.ndarray:
    U = new_field(dims)
    lib().orc_init_links(_dp(U.view(np.float64)), _dims(dims), int(start), seed, lattice_id)
    return U


def plaquette(U, dims) -> float:
    return float(lib().orc_plaquette(_dp(U.view(np.float64)), _dims(dims)))


def action(U, dims, beta) -> float:
    return float(lib().orc_action(_dp(U.view(np.float64)), _dims(dims), float(beta)))


def staple(U, dims, s, mu) -> np.ndarray:
    A = np.zeros((3, 3), dtype=np.complex128)
    lib().orc_staple(_dp(U.view(np.float64)), _dims(dims), int(s), int(mu), _dp(A.view(np.float64)))
    return A


def creutz_samples(k, seed, n):
    x = np.zeros((n, 4))
    acc = np.zeros(n, dtype=np.int32)
    lib().orc_creutz_samples(float(k), seed, int(n), _dp(x), acc.ctypes.data_as(_I))
    return x, acc


def or_link_ordered(Ul, A, order):
    out = np.zeros((3, 3), dtype=np.complex128)
    Ul = np.ascontiguousarray(Ul, dtype=np.complex128)
    A = np.ascontiguousarray(A, dtype=np.complex128)
    o = (ctypes.c_int * 3)(*order)
    lib().orc_or_link_ordered(_dp(Ul.view(np.float64)), _dp(A.view(np.float64)), o, _dp(out.view(np.float64)))
    return out


def _dec_ptr(dec):
    return None if dec is None else dec.ctypes.data_as(_U8)


def new_decisions(dims) -> np.ndarray:
    return np.full((volume(dims), 4, 3), 255, dtype=np.uint8)


def heatbath_sweep(U, dims, beta, seed, lattice_id, sweep, n_hb=1, dec=None):
    lib().orc_heatbath_sweep(_dp(U.view(np.float64)), _dims(dims), float(beta), seed, lattice_id, sweep,
                             int(n_hb), _dec_ptr(dec))


def heatbath_subsweep(U, dims, beta, seed, lattice_id, sweep, n_hb, mu, parity, dec=None):
    lib().orc_heatbath_subsweep(_dp(U.view(np.float64)), _dims(dims), float(beta), seed, lattice_id, sweep,
                                int(n_hb), int(mu), int(parity), _dec_ptr(dec))


def heatbath_one_link(U, dims, beta, seed, lattice_id, sweep, n_hb, s, mu):
    out = np.zeros((3, 3), dtype=np.complex128)
    dec = np.zeros(3, dtype=np.uint8)
    lib().orc_heatbath_one_link(_dp(U.view(np.float64)), _dims(dims), float(beta), seed, lattice_id, sweep,
                                int(n_hb), int(s), int(mu), _dp(out.view(np.float64)), dec.ctypes.data_as(_U8))
    return out, dec


def heatbath_link_staple(Ul, A, beta, seed, lattice_id, sweep, n_hb, s, mu):
    """Heat-bath result for link Ul (3x3) with staple A (3x3) at lexicographic
    site s, direction mu: heatbath_one_link without the lattice."""
    out = np.zeros((3, 3), dtype=np.complex128)
    dec = np.zeros(3, dtype=np.uint8)
    Ul = np.ascontiguousarray(Ul, dtype=np.complex128)
    A = np.ascontiguousarray(A, dtype=np.complex128)
    lib().orc_heatbath_link_staple(_dp(Ul.view(np.float64)), _dp(A.view(np.float64)), float(beta), seed,
                                   lattice_id, sweep, int(n_hb), int(s), int(mu), _dp(out.view(np.float64)),
                                   dec.ctypes.data_as(_U8))
    return out, dec


def overrelax_sweep(U, dims):
    lib().orc_overrelax_sweep(_dp(U.view(np.float64)), _dims(dims))


def overrelax_subsweep(U, dims, mu, parity):
    lib().orc_overrelax_subsweep(_dp(U.view(np.float64)), _dims(dims), int(mu), int(parity))


def subsweep_range(U, dims, kind, beta, seed, lattice_id, sweep, n_hb, mu, parity, s_lo, s_hi):
    """(mu, parity) heat-bath (kind 0) or overrelaxation (kind 1) updates of the sites in [s_lo, s_hi)."""
    lib().orc_subsweep_range(_dp(U.view(np.float64)), _dims(dims), int(kind), float(beta), seed, lattice_id, sweep,
                             int(n_hb), int(mu), int(parity), int(s_lo), int(s_hi))


def overrelax_one_link(U, dims, s, mu):
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().orc_overrelax_one_link(_dp(U.view(np.float64)), _dims(dims), int(s), int(mu), _dp(out.view(np.float64)))
    return out


def update_chain(U, dims, beta, seed, lattice_id, sweep0, n_sweeps, n_hb=1, n_or=4):
    plaq = np.zeros(n_sweeps)
    lib().orc_update_chain(_dp(U.view(np.float64)), _dims(dims), float(beta), seed, lattice_id, sweep0,
                           int(n_sweeps), int(n_hb), int(n_or), _dp(plaq))
    return plaq


# ---------------------------------------------------------------- algebra
def expm(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.complex128)
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().orc_expm(_dp(X.view(np.float64)), _dp(out.view(np.float64)))
    return out


def alg_to_mat(p) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().orc_alg_to_mat(_dp(p), _dp(out.view(np.float64)))
    return out


def mat_to_alg(M) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.complex128)
    p = np.zeros(8)
    lib().orc_mat_to_alg(_dp(M.view(np.float64)), _dp(p))
    return p


def su3_project(M, n_pass=8) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.complex128)
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().orc_su3_project(_dp(M.view(np.float64)), int(n_pass), _dp(out.view(np.float64)))
    return out


def reunit(M) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.complex128)
    out = np.zeros((3, 3), dtype=np.complex128)
    lib().orc_reunit(_dp(M.view(np.float64)), _dp(out.view(np.float64)))
    return out


# ---------------------------------------------------------------- HMC
def force(U, dims, beta) -> np.ndarray:
    F = np.zeros((volume(dims), 4, 8))
    lib().orc_force(_dp(U.view(np.float64)), _dims(dims), float(beta), _dp(F))
    return F


def mom_refresh(dims, seed, lattice_id, traj) -> np.ndarray:
    P = np.zeros((volume(dims), 4, 8))
    lib().orc_mom_refresh(_dp(P), _dims(dims), seed, lattice_id, traj)
    return P


def kinetic(P, dims) -> float:
    return float(lib().orc_kinetic(_dp(P), _dims(dims)))


def update_links(U, P, dims, eps):
    lib().orc_update_links(_dp(U.view(np.float64)), _dp(P), _dims(dims), float(eps))


def leapfrog(U, P, dims, beta, tau, n_steps):
    lib().orc_leapfrog(_dp(U.view(np.float64)), _dp(P), _dims(dims), float(beta), float(tau), int(n_steps))


def hmc_trajectory(U, dims, beta, tau, n_steps, seed, lattice_id, traj, accept_reject=1, P=None):
    if P is None:
        P = np.zeros((volume(dims), 4, 8))
    dH = ctypes.c_double()
    acc = ctypes.c_int()
    lib().orc_hmc_trajectory(_dp(U.view(np.float64)), _dp(P), _dims(dims), float(beta), float(tau),
                             int(n_steps), seed, lattice_id, traj, int(accept_reject), ctypes.byref(dH),
                             ctypes.byref(acc))
    return float(dH.value), int(acc.value)


# ---------------------------------------------------------------- multiscale
def restrict(Uf, dims_f) -> np.ndarray:
    dc = [int(v) // 2 for v in dims_f]
    Uc = new_field(dc)
    lib().orc_restrict(_dp(Uf.view(np.float64)), _dims(dims_f), _dp(Uc.view(np.float64)))
    return Uc


def transfer(Uc, dims_c) -> np.ndarray:
    df = [2 * int(v) for v in dims_c]
    Uf = new_field(df)
    lib().orc_transfer(_dp(Uc.view(np.float64)), _dims(dims_c), _dp(Uf.view(np.float64)))
    return Uf


def partial_action(U, dims, d) -> float:
    return float(lib().orc_partial_action(_dp(U.view(np.float64)), _dims(dims), int(d)))


def ape_step(U, dims, d, c=0.05, n_pass=8) -> np.ndarray:
    """One Jacobi APE step of interpolation stage d on a copy of U (Eq. APE)."""
    W = np.ascontiguousarray(U.copy())
    lib().orc_ape_step(_dp(W.view(np.float64)), _dims(dims), int(d), float(c), int(n_pass))
    return W


def prolongate(Uc, dims_c, c=0.05, rel_tol=1e-5, max_iter=10000, n_pass=8):
    df = [2 * int(v) for v in dims_c]
    Uf = new_field(df)
    iters = (ctypes.c_int * 3)()
    sd = np.zeros(3)
    lib().orc_prolongate(_dp(Uc.view(np.float64)), _dims(dims_c), _dp(Uf.view(np.float64)), float(c),
                         float(rel_tol), int(max_iter), int(n_pass), iters, _dp(sd))
    return Uf, [int(v) for v in iters], sd


# ---------------------------------------------------------------- flow
def flow_step(W, dims, eps):
    lib().orc_flow_step(_dp(W.view(np.float64)), _dims(dims), float(eps))


def clover_EQ(U, dims):
    E = ctypes.c_double()
    Q = ctypes.c_double()
    lib().orc_clover_EQ(_dp(U.view(np.float64)), _dims(dims), ctypes.byref(E), ctypes.byref(Q))
    return float(E.value), float(Q.value)


def clover_q_site(U, dims, s, m) -> float:
    """Clover charge density at site s from the m x m leaves (no 1/m^4); m = 0:
    the three-loop improved density."""
    return float(lib().orc_clover_q_site(_dp(U.view(np.float64)), _dims(dims), int(s), int(m)))


def topo_charge_improved(U, dims) -> np.ndarray:
    """[Q_improved, Q_1x1, Q_2x2, Q_3x3] (Sec. IV.C, three-loop improved charge)."""
    out = np.zeros(4)
    lib().orc_topo_charge_improved(_dp(U.view(np.float64)), _dims(dims), _dp(out))
    return out


def wilson_flow_times(W, dims, t_end, eps, t_meas, charge=0):
    """Flow W in place to t_end (steps eps, shortened to land on each t_meas);
    returns E, Q at t_meas (charge 0: clover Q, 1: improved Q)."""
    tm = np.ascontiguousarray(np.asarray(t_meas, dtype=np.float64))
    E, Q = np.zeros(tm.size), np.zeros(tm.size)
    lib().orc_wilson_flow_times(_dp(W.view(np.float64)), _dims(dims), float(t_end), float(eps), _dp(tm), int(tm.size),
                                int(charge), _dp(E), _dp(Q))
    return E, Q


def wilson_flow(W, dims, eps, n_steps, meas_every):
    m = n_steps // meas_every + 1
    E = np.zeros(m)
    Q = np.zeros(m)
    lib().orc_wilson_flow(_dp(W.view(np.float64)), _dims(dims), float(eps), int(n_steps), int(meas_every),
                          _dp(E), _dp(Q))
    return E, Q


def flow_trial_step(W, dims, h) -> float:
    """One adaptive-flow trial step of size h (kept); returns the error d."""
    return float(lib().orc_flow_trial_step(_dp(W.view(np.float64)), _dims(dims), float(h)))


def adaptive_measurements(t_end, dt_meas) -> int:
    """Measurement times k dt_meas <= t_end, plus t_end if it is not one."""
    k = int(np.floor(t_end / dt_meas + 1e-9))
    return k + 1 + (1 if t_end - k * dt_meas > 1e-12 * dt_meas else 0)


def wilson_flow_adaptive(W, dims, t_end, tol, eps_max, eps0, dt_meas):
    """Adaptive-step flow to t_end; returns (E, Q, steps, rejects)."""
    m = adaptive_measurements(t_end, dt_meas)
    E = np.zeros(m)
    Q = np.zeros(m)
    steps, rejects = ctypes.c_int(0), ctypes.c_int(0)
    got = lib().orc_wilson_flow_adaptive(_dp(W.view(np.float64)), _dims(dims), float(t_end), float(tol),
                                         float(eps_max), float(eps0), float(dt_meas), _dp(E), _dp(Q), m,
                                         ctypes.byref(steps), ctypes.byref(rejects))
    return E[:got], Q[:got], steps.value, rejects.value


# ---------------------------------------------------------------- loops
def wilson_loop(U, dims, m, n) -> float:
    return float(lib().orc_wilson_loop(_dp(U.view(np.float64)), _dims(dims), int(m), int(n)))


def partial_loops(U, dims) -> np.ndarray:
    """[W1x1_0..2, W2x2_0..4, h] (see orc_partial_loops)."""
    out = np.zeros(9)
    lib().orc_partial_loops(_dp(U.view(np.float64)), _dims(dims), _dp(out))
    return out
