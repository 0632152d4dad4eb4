"""Python face of libmgq: the same entry points as include/mgq.h, taking a
:class:`Lattice` whose device buffers are torch tensors.  Only argument
marshalling happens here; every step of the hot path runs in the CUDA
kernels of libmgq."""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import MGQ_F32, MGQ_F32_C12, MGQ_F64, MgqError, MgqLattice, call

PRECISIONS = {"f64": MGQ_F64, "f32": MGQ_F32, "f32c12": MGQ_F32_C12}


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Lattice:
    """One lattice: extents, precision, RNG key and its device buffers.

    links / work (and mom, when ``with_mom``) are uint8 torch tensors of the
    sizes the library asks for; the struct handed to the C ABI points into
    them.
    """

    def __init__(self, dims: Sequence[int], prec: str = "f64", seed: int = 0, lattice_id: int = 0,
                 with_mom: bool = False, device: str | torch.device = "cuda"):
        self.dims = [int(v) for v in dims]
        self.prec = prec
        self.device = torch.device(device)
        c = MgqLattice()
        for m in range(4):
            c.dims[m] = self.dims[m]
            c.bc[m] = 0
        c.prec = PRECISIONS[prec]
        c.action = 0
        c.seed = int(seed)
        c.lattice_id = int(lattice_id)
        c.reserved = 0
        L = _lib.load()
        nl = int(L.mgq_links_bytes(ctypes.byref(c)))
        if nl == 0:
            raise MgqError(_lib.MGQ_EINVAL, f"invalid extents {self.dims} for prec {prec}")
        nw = int(L.mgq_workspace_bytes(ctypes.byref(c)))
        nm = int(L.mgq_mom_bytes(ctypes.byref(c)))
        self.links = torch.zeros(nl, dtype=torch.uint8, device=self.device)
        self.work = torch.zeros(nw, dtype=torch.uint8, device=self.device)
        self.mom = torch.zeros(nm, dtype=torch.uint8, device=self.device) if with_mom else None
        c.links = self.links.data_ptr()
        c.work = self.work.data_ptr()
        c.work_bytes = nw
        c.mom = self.mom.data_ptr() if self.mom is not None else None
        self.c = c
        self.volume = int(np.prod(self.dims))
        self.site_stride = int(L.mgq_site_stride((ctypes.c_int32 * 4)(*self.dims)))

    @property
    def ref(self):
        return ctypes.byref(self.c)

    @property
    def seed(self) -> int:
        return int(self.c.seed)

    @property
    def lattice_id(self) -> int:
        return int(self.c.lattice_id)

    def real_dtype(self) -> torch.dtype:
        return torch.float64 if self.prec == "f64" else torch.float32

    def new_alg_field(self) -> torch.Tensor:
        """A zeroed device buffer in the momentum layout (4*2*8*S reals)."""
        return torch.zeros(4 * 2 * 8 * self.site_stride, dtype=self.real_dtype(), device=self.device)

    # ---------------------------------------------------------- canonical I/O
    def to_numpy(self, stream=None) -> np.ndarray:
        """Export the links as complex128 (V, 4, 3, 3) in lexicographic site order."""
        buf = torch.empty(self.volume * 72, dtype=torch.float64, device=self.device)
        mgq_export_links(self, buf, stream)
        return buf.cpu().numpy().view(np.complex128).reshape(self.volume, 4, 3, 3)

    def from_numpy(self, U: np.ndarray, stream=None) -> None:
        """Import links given as complex128 (V, 4, 3, 3) in lexicographic site order."""
        a = np.ascontiguousarray(U, dtype=np.complex128).view(np.float64).reshape(-1)
        buf = torch.from_numpy(a.copy()).to(self.device)
        mgq_import_links(self, buf, stream)
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def mom_numpy(self) -> np.ndarray:
        """Momenta as float64 (V, 4, 8) in lexicographic site order."""
        return alg_to_numpy(self, self.mom)


def _alg_blocks(lat: Lattice, buf: torch.Tensor) -> torch.Tensor:
    """A view of an algebra buffer as [mu][parity][h/32][a][h%32] (the device layout)."""
    S = lat.site_stride
    return buf.view(lat.real_dtype()).reshape(4, 2, S // 32, 8, 32)


def _site_index(lat: Lattice):
    """Parity and half index h of every lexicographic site."""
    L = lat.dims
    idx = np.arange(lat.volume)
    x = [(idx // int(np.prod(L[:m]))) % L[m] for m in range(4)]
    return (x[0] + x[1] + x[2] + x[3]) % 2, idx // 2


def alg_to_numpy(lat: Lattice, buf: torch.Tensor) -> np.ndarray:
    """A buffer in the momentum layout, as float64 (V, 4, 8) in lexicographic site order."""
    a = _alg_blocks(lat, buf).double().cpu().numpy()
    par, h = _site_index(lat)
    out = np.empty((lat.volume, 4, 8))
    for mu in range(4):
        out[:, mu, :] = a[mu, par, h // 32, :, h % 32]
    return out


def alg_from_numpy(lat: Lattice, P: np.ndarray) -> torch.Tensor:
    """A device buffer in the momentum layout from float64 (V, 4, 8) in lexicographic site order."""
    a = np.zeros((4, 2, lat.site_stride // 32, 8, 32))
    par, h = _site_index(lat)
    for mu in range(4):
        a[mu, par, h // 32, :, h % 32] = P[:, mu, :]
    return torch.from_numpy(a.reshape(-1)).to(device=lat.device, dtype=lat.real_dtype())


def zero_alg_padding(lat: Lattice, buf: torch.Tensor) -> None:
    """Zero the entries of the padding sites h >= V/2 (which carry no links)."""
    h = torch.arange(lat.volume // 2, lat.site_stride, device=buf.device)
    _alg_blocks(lat, buf)[:, :, h // 32, :, h % 32] = 0


# ------------------------------------------------------------------ entry points
def mgq_init_links(lat: Lattice, start: int, stream=None) -> None:
    call("mgq_init_links", lat.ref, int(start), _stream_handle(stream))


def mgq_import_links(lat: Lattice, canon: torch.Tensor, stream=None) -> None:
    call("mgq_import_links", lat.ref, _ptr(canon), _stream_handle(stream))


def mgq_export_links(lat: Lattice, canon: torch.Tensor, stream=None) -> None:
    call("mgq_export_links", lat.ref, _ptr(canon), _stream_handle(stream))


def mgq_heatbath_sweep(lat: Lattice, beta: float, sweep: int, n_hb: int = 1, stream=None) -> None:
    call("mgq_heatbath_sweep", lat.ref, float(beta), int(sweep), int(n_hb), _stream_handle(stream))


def mgq_heatbath_subsweep(lat: Lattice, beta: float, sweep: int, n_hb: int, mu: int, parity: int,
                          decisions: Optional[torch.Tensor] = None, stream=None) -> None:
    call("mgq_heatbath_subsweep", lat.ref, float(beta), int(sweep), int(n_hb), int(mu), int(parity),
         _ptr(decisions), _stream_handle(stream))


def mgq_overrelax_sweep(lat: Lattice, stream=None) -> None:
    call("mgq_overrelax_sweep", lat.ref, _stream_handle(stream))


def mgq_overrelax_sweep_plaquette(lat: Lattice, out=None, stream=None) -> Optional[float]:
    """One overrelaxation sweep that also measures the plaquette of the result;
    into `out` (device tensor) or returned as a float."""
    if out is not None:
        call("mgq_overrelax_sweep_plaquette", lat.ref, _ptr(out), _stream_handle(stream))
        return None
    v = ctypes.c_double()
    call("mgq_overrelax_sweep_plaquette", lat.ref, ctypes.byref(v), _stream_handle(stream))
    return float(v.value)


def mgq_update_sweeps(lat: Lattice, beta: float, sweep0: int, n_sweeps: int, n_hb: int = 1, n_or: int = 4,
                      plaq_out=None, stream=None):
    """n_sweeps x (1 HB + n_or OR); returns the per-sweep plaquettes when plaq_out is True or a tensor."""
    out = None
    if plaq_out is True:
        out = np.zeros(n_sweeps)
        ptr = ctypes.c_void_p(out.ctypes.data)
    elif isinstance(plaq_out, torch.Tensor):
        ptr = _ptr(plaq_out)
    elif isinstance(plaq_out, np.ndarray):
        out = plaq_out
        ptr = ctypes.c_void_p(plaq_out.ctypes.data)
    else:
        ptr = None
    call("mgq_update_sweeps", lat.ref, float(beta), int(sweep0), int(n_sweeps), int(n_hb), int(n_or), ptr,
         _stream_handle(stream))
    return out


def mgq_plaquette(lat: Lattice, out=None, stream=None) -> Optional[float]:
    """Average plaquette; into `out` (device tensor) or returned as a float."""
    if out is not None:
        call("mgq_plaquette", lat.ref, _ptr(out), _stream_handle(stream))
        return None
    v = ctypes.c_double()
    call("mgq_plaquette", lat.ref, ctypes.byref(v), _stream_handle(stream))
    return float(v.value)


def mgq_topo_charge(lat: Lattice, stream=None):
    E, Q = ctypes.c_double(), ctypes.c_double()
    call("mgq_topo_charge", lat.ref, ctypes.byref(E), ctypes.byref(Q), _stream_handle(stream))
    return float(E.value), float(Q.value)


def mgq_topo_charge_improved(lat: Lattice, stream=None) -> np.ndarray:
    """[Q_improved, Q_1x1, Q_2x2, Q_3x3]: the three-loop improved charge and its m x m clover parts."""
    out = np.zeros(4)
    call("mgq_topo_charge_improved", lat.ref, ctypes.c_void_p(out.ctypes.data), _stream_handle(stream))
    return out


def mgq_wilson_flow_times(lat: Lattice, t_end: float, eps: float, t_meas, charge: str = "clover", stream=None):
    """Flow to t_end with steps eps shortened to land on every t_meas; returns E, Q at t_meas.
    charge: "clover" or "improved" (three-loop improved Q)."""
    tm = np.ascontiguousarray(np.asarray(t_meas, dtype=np.float64))
    E, Q = np.zeros(tm.size), np.zeros(tm.size)
    call("mgq_wilson_flow_times", lat.ref, float(t_end), float(eps), ctypes.c_void_p(tm.ctypes.data), int(tm.size),
         {"clover": 0, "improved": 1}[charge], ctypes.c_void_p(E.ctypes.data), ctypes.c_void_p(Q.ctypes.data),
         _stream_handle(stream))
    return E, Q


def mgq_wilson_flow(lat: Lattice, eps: float, n_steps: int, meas_every: int, stream=None):
    m = n_steps // meas_every + 1
    E, Q = np.zeros(m), np.zeros(m)
    call("mgq_wilson_flow", lat.ref, float(eps), int(n_steps), int(meas_every), ctypes.c_void_p(E.ctypes.data),
         ctypes.c_void_p(Q.ctypes.data), _stream_handle(stream))
    return E, Q


def mgq_wilson_flow_adaptive(lat: Lattice, t_end: float, tol: float = 0.01, eps_max: float = 0.2,
                             eps0: float = 0.01, dt_meas: float | None = None, stream=None):
    """Adaptive-step flow to t_end; returns (E, Q, steps, rejects), E and Q at
    t = k dt_meas <= t_end and at t_end (dt_meas defaults to t_end)."""
    dt = float(t_end if dt_meas is None else dt_meas)
    L = _lib.load()
    m = int(L.mgq_flow_adaptive_measurements(float(t_end), dt))
    if m < 0:
        raise ValueError("mgq_wilson_flow_adaptive: need t_end >= 0 and dt_meas > 0")
    n = int(L.mgq_flow_adaptive_scratch_bytes(lat.ref))
    scratch = torch.empty(n, dtype=torch.uint8, device=lat.device)
    E, Q = np.zeros(m), np.zeros(m)
    nm, ns, nr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    call("mgq_wilson_flow_adaptive", lat.ref, float(t_end), float(tol), float(eps_max), float(eps0), dt,
         ctypes.c_void_p(E.ctypes.data), ctypes.c_void_p(Q.ctypes.data), ctypes.byref(nm), ctypes.byref(ns),
         ctypes.byref(nr), _ptr(scratch), n, _stream_handle(stream))
    return E[:nm.value], Q[:nm.value], int(ns.value), int(nr.value)


def mgq_hmc_force(lat: Lattice, beta: float, force_out: torch.Tensor, stream=None) -> None:
    call("mgq_hmc_force", lat.ref, float(beta), _ptr(force_out), _stream_handle(stream))


def mgq_hmc_trajectory(lat: Lattice, beta: float, tau: float, n_steps: int, traj: int, accept_reject: int = 1,
                       stream=None):
    dH, acc = ctypes.c_double(), ctypes.c_int()
    call("mgq_hmc_trajectory", lat.ref, float(beta), float(tau), int(n_steps), int(traj), int(accept_reject),
         ctypes.byref(dH), ctypes.byref(acc), _stream_handle(stream))
    return float(dH.value), int(acc.value)


def mgq_prolongate(coarse: Lattice, fine: Lattice, c: float = 0.05, rel_tol: float = 1e-5, max_iter: int = 10000,
                   stream=None):
    iters = (ctypes.c_int * 3)()
    sd = (ctypes.c_double * 3)()
    call("mgq_prolongate", coarse.ref, fine.ref, float(c), float(rel_tol), int(max_iter), iters, sd,
         _stream_handle(stream))
    return [int(v) for v in iters], [float(v) for v in sd]


class ProlongBatch:
    """Lattice pairs (coarse -> fine) prolongated together by mgq_prolongate_batched.

    The descriptor arrays, the work buffer and the device result buffers are
    built once, so repeated calls (and CUDA-graph capture) pass the same pointers.
    """

    def __init__(self, coarse: Sequence[Lattice], fine: Sequence[Lattice]):
        if len(coarse) != len(fine) or not fine:
            raise ValueError("need one fine lattice per coarse lattice")
        self.coarse, self.fine = list(coarse), list(fine)
        self.n = len(self.fine)
        self.carr = (MgqLattice * self.n)(*[l.c for l in self.coarse])
        self.farr = (MgqLattice * self.n)(*[l.c for l in self.fine])
        nb = int(_lib.load().mgq_prolongate_batched_workspace_bytes(self.farr, self.n))
        if nb == 0:
            raise MgqError(_lib.MGQ_EINVAL, "invalid lattice extents in prolongation batch")
        dev = self.fine[0].device
        self.work = torch.zeros(nb, dtype=torch.uint8, device=dev)
        self.iters = torch.zeros((self.n, 3), dtype=torch.int32, device=dev)
        self.sd = torch.zeros((self.n, 3), dtype=torch.float64, device=dev)
        self.n_done = torch.zeros(1, dtype=torch.int32, device=dev)


def mgq_prolongate_batched(batch: ProlongBatch, c: float = 0.05, rel_tol: float = 1e-5, max_iter: int = 10000,
                           iter_budget: int = 0, stream=None) -> None:
    """Prolongate every pair of the batch; results land in batch.iters, batch.sd
    (device, per lattice) and batch.n_done.  iter_budget > 0: exactly that many
    APE iterations, no host synchronisation (graph-capturable)."""
    call("mgq_prolongate_batched", batch.carr, batch.farr, batch.n, float(c), float(rel_tol), int(max_iter),
         int(iter_budget), _ptr(batch.iters), _ptr(batch.sd), _ptr(batch.n_done), _ptr(batch.work),
         int(batch.work.numel()), _stream_handle(stream))


def mgq_restrict(fine: Lattice, coarse: Lattice, stream=None) -> None:
    call("mgq_restrict", fine.ref, coarse.ref, _stream_handle(stream))


def mgq_reunitarize(lat: Lattice, fp64_projection: bool = False, stream=None) -> None:
    """Gram-Schmidt projection of every link onto SU(3) (FP32 formats: in FP32 or FP64)."""
    call("mgq_reunitarize", lat.ref, int(bool(fp64_projection)), _stream_handle(stream))


def mgq_check_unitarity(lat: Lattice, tol: float = 0.0, stream=None) -> float:
    v = ctypes.c_double()
    call("mgq_check_unitarity", lat.ref, float(tol), ctypes.byref(v), _stream_handle(stream))
    return float(v.value)


# ------------------------------------------------------------------ batched driver
class Batch:
    """Independent lattices advanced together by mgq_update_sweeps_batched.

    The ctypes array of their descriptors and the batch workspace (sized for
    ``max_sweeps`` plaquette records) are built once, so repeated calls (and
    CUDA-graph capture of them) pass the same pointers.
    """

    def __init__(self, lattices: Sequence[Lattice], betas: Sequence[float], max_sweeps: int = 64):
        if len(lattices) != len(betas) or not lattices:
            raise ValueError("need one beta per lattice")
        self.lattices = list(lattices)
        self.n = len(self.lattices)
        self.arr = (MgqLattice * self.n)(*[l.c for l in self.lattices])
        self.betas = (ctypes.c_double * self.n)(*[float(b) for b in betas])
        self.max_sweeps = int(max_sweeps)
        nb = int(_lib.load().mgq_batch_workspace_bytes(self.arr, self.n, self.max_sweeps))
        if nb == 0:
            raise MgqError(_lib.MGQ_EINVAL, "invalid lattice extents in batch")
        self.work = torch.zeros(nb, dtype=torch.uint8, device=self.lattices[0].device)

    def plaquette_buffer(self, n_sweeps: int) -> torch.Tensor:
        return torch.zeros((n_sweeps, self.n), dtype=torch.float64, device=self.lattices[0].device)


def mgq_update_sweeps_batched(batch: Batch, sweep0: int, n_sweeps: int, n_hb: int = 1, n_or: int = 4,
                              plaq_out: Optional[torch.Tensor] = None, stream=None) -> None:
    """n_sweeps compound sweeps on every lattice of the batch; plaq_out: device (n_sweeps, n) float64 or None."""
    if plaq_out is not None and n_sweeps > batch.max_sweeps:
        raise ValueError("batch workspace sized for fewer sweeps")
    call("mgq_update_sweeps_batched", batch.arr, batch.n, batch.betas, int(sweep0), int(n_sweeps), int(n_hb),
         int(n_or), _ptr(plaq_out), _ptr(batch.work), int(batch.work.numel()), _stream_handle(stream))


def mgq_hmc_momentum_step(lat: Lattice, beta: float, eps: float, stream=None) -> None:
    """P <- P + eps F(U) on lat.mom: the leapfrog's fused force + P-step."""
    call("mgq_hmc_momentum_step", lat.ref, float(beta), float(eps), _stream_handle(stream))


def fma_probe(iters: int, sink: torch.Tensor, stream=None) -> int:
    """Launch the FP32 FMA probe; returns the launch's floating-point operations."""
    return int(_lib.load().mgq_fma_probe(int(iters), _ptr(sink), _stream_handle(stream)))


def mgq_link_exp_update(lat: Lattice, alg: torch.Tensor, s: float = 1.0, stream=None) -> None:
    """U <- exp(s P) U on every link, P from an algebra field in the momentum layout."""
    call("mgq_link_exp_update", lat.ref, _ptr(alg), float(s), _stream_handle(stream))


def copy_lattice(lat: Lattice, with_mom: bool = False) -> Lattice:
    """A new lattice with the same extents, precision, RNG key and a copy of the links."""
    c = Lattice(lat.dims, lat.prec, seed=lat.seed, lattice_id=lat.lattice_id, with_mom=with_mom, device=lat.device)
    c.links.copy_(lat.links)
    return c


# ------------------------------------------------------------------ checkpoints
_MAGIC = b"MGQCKPT3"  # 3: links in 32-site blocks of planes, FP32 12-real as 16-byte plane pairs


def save_checkpoint(lat: Lattice, path: str, beta: float, sweep: int) -> None:
    """Raw little-endian dump of the link buffer with a header (extents, precision,
    seed, lattice id, beta, next sweep index) and a CRC-32 of the payload.  The
    RNG is counter-based, so continuing from `sweep` reproduces the
    uninterrupted chain bit for bit."""
    import struct
    import zlib

    torch.cuda.synchronize()
    payload = lat.links.cpu().numpy().tobytes()
    hdr = struct.pack("<8s4iiQIdQQI", _MAGIC, *lat.dims, PRECISIONS[lat.prec], lat.seed, lat.lattice_id, float(beta),
                      int(sweep), len(payload), zlib.crc32(payload) & 0xFFFFFFFF)
    with open(path, "wb") as f:
        f.write(hdr)
        f.write(payload)


def load_checkpoint(path: str, device="cuda"):
    """Returns (lattice, beta, sweep); raises ValueError on a corrupted file."""
    import struct
    import zlib

    fmt = "<8s4iiQIdQQI"
    with open(path, "rb") as f:
        raw = f.read()
    n = struct.calcsize(fmt)
    magic, d0, d1, d2, d3, prec, seed, lid, beta, sweep, nbytes, crc = struct.unpack(fmt, raw[:n])
    payload = raw[n:]
    if magic != _MAGIC or len(payload) != nbytes or (zlib.crc32(payload) & 0xFFFFFFFF) != crc:
        raise ValueError(f"{path}: not an intact mgq checkpoint")
    name = {v: k for k, v in PRECISIONS.items()}[prec]
    lat = Lattice([d0, d1, d2, d3], name, seed=seed, lattice_id=lid, device=device)
    if lat.links.numel() != nbytes:
        raise ValueError(f"{path}: payload size does not match the lattice layout")
    lat.links.copy_(torch.frombuffer(bytearray(payload), dtype=torch.uint8))
    return lat, beta, sweep


# ------------------------------------------------------------------ adjoint flow
def mgq_flow_vjp(lat: Lattice, psi: torch.Tensor, scale: float, lam: torch.Tensor, stream=None) -> None:
    """lam += scale * DZ(W)^T psi for the flow generator Z(W) = -TA(W A(W)) at the lattice's links."""
    call("mgq_flow_vjp", lat.ref, _ptr(psi), float(scale), _ptr(lam), _stream_handle(stream))


def mgq_exp_vjp(lat: Lattice, omega: torch.Tensor, g_in: torch.Tensor, g_out: torch.Tensor, stream=None) -> None:
    """g_out = J(omega)^T g_in: a cotangent at exp(omega) U pulled back to omega."""
    call("mgq_exp_vjp", lat.ref, _ptr(omega), _ptr(g_in), _ptr(g_out), _stream_handle(stream))


def flow_adjoint_scratch(lat: Lattice) -> torch.Tensor:
    n = int(_lib.load().mgq_flow_adjoint_scratch_bytes(lat.ref))
    return torch.zeros(n, dtype=torch.uint8, device=lat.device)


def mgq_wilson_flow_step_adjoint(lat: Lattice, eps: float, lam: torch.Tensor, scratch: torch.Tensor,
                                 stream=None) -> None:
    """Pull a cotangent back through one RK3 flow step that starts at the lattice's links."""
    call("mgq_wilson_flow_step_adjoint", lat.ref, float(eps), _ptr(lam), _ptr(scratch), int(scratch.numel()),
         _stream_handle(stream))


# ------------------------------------------------------------------ loops
def mgq_wilson_loop(lat: Lattice, m: int, n: int, stream=None) -> float:
    v = ctypes.c_double()
    call("mgq_wilson_loop", lat.ref, int(m), int(n), ctypes.byref(v), _stream_handle(stream))
    return float(v.value)


def mgq_partial_loops(lat: Lattice, stream=None) -> np.ndarray:
    """[W1x1_0..2, W2x2_0..4, h] as float64."""
    out = np.zeros(9)
    call("mgq_partial_loops", lat.ref, ctypes.c_void_p(out.ctypes.data), _stream_handle(stream))
    return out


def mgq_clover_vjp(lat: Lattice, observable: str, scale: float, lam: torch.Tensor, stream=None) -> None:
    """lam += scale * gradient of the clover observable ("E" or "Q") at the lattice's links."""
    n = int(_lib.load().mgq_clover_vjp_scratch_bytes(lat.ref))
    scratch = torch.empty(n, dtype=torch.uint8, device=lat.device)
    call("mgq_clover_vjp", lat.ref, {"E": 0, "Q": 1}[observable], float(scale), _ptr(lam), _ptr(scratch), n,
         _stream_handle(stream))
