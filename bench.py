#!/usr/bin/env python
"""Throughput of the multiscale-thermalization hot path on GB300.

Workload (one step): one compound sweep of a 32^4 SU(3) Wilson lattice at
beta = 6.0 -- one Cabibbo-Marinari heat-bath sweep (N_hb = 1) followed by
four overrelaxation sweeps on the checkerboard schedule -- plus the FP64
average plaquette of the result, as the rethermalisation stage of the
multiscale method runs it.  Links are FP32 with 12-real (two-row)
compression; reductions are FP64.  The value is link updates per second
over the whole job (5 x 4V updates per step per GPU).

Also measured in the same run: the HMC gauge force + momentum update in
algorithmic GB/s, the plain FP64 GPU path and the 18-real FP32 path
(link updates/s), an end-to-end number through the C ABI with the step's
input links copied from pinned host memory and the plaquette read back,
and the FP64 CPU oracle on a bounded sample (cpu_baseline).

Multi-GPU: replicas only (independent lattices, one per rank; no
collective on the data path).  `--impl reference` times the CPU oracle.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "link updates/s + force GB/s, 32^4 SU(3), vs plain FP64 GPU; % HBM roofline"
UNIT = "link updates/s"
LINK_BYTES = {"f64": 144, "f32": 72, "f32c12": 48}
REAL_BYTES = {"f64": 8, "f32": 4, "f32c12": 4}
# FP32 ALU peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2.07 GHz
# (a packed FFMA2 issues at half rate, so it does not raise this).  FP64 on this part is far lower.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic real flops per link (complex multiply 6, complex add 2, 3x3 complex product 198):
# staple = 12 products + 5 matrix sums = 2466; the force adds U.A (198) and the traceless
# antihermitian projection and scaled accumulate (36); the overrelaxation adds U.A (198), three
# SU(2) subgroup steps (about 200 each) and the reunitarisation (about 140); the heat bath adds
# the Creutz sampler (about 60 per subgroup) to that.
FLOPS_PER_LINK = {"k_force": 2700, "k_overrelax": 3400, "k_heatbath": 3580}


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["mgq", "reference"], default="mgq")
    p.add_argument("--prec", choices=["f64", "f32", "f32c12"], default="f32c12")
    p.add_argument("--dims", default="32,32,32,32")
    p.add_argument("--beta", type=float, default=6.0)
    p.add_argument("--n-or", type=int, default=4)
    p.add_argument("--therm", type=int, default=30, help="untimed thermalisation sweeps before timing")
    p.add_argument("--no-extras", action="store_true", help="skip the FP64/FP32 comparison legs")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--large", action="store_true", help="add the 48^4 FP32/FP64 leg")
    return p.parse_args()


def workload_config(args, dims):
    V = 1
    for d in dims:
        V *= d
    return {
        "workload": f"{'x'.join(map(str, dims))} SU(3) Wilson beta={args.beta}: 1 heat-bath (Creutz, N_hb=1) + "
                    f"{args.n_or} overrelaxation sweeps + FP64 plaquette per step",
        "lattice": dims,
        "beta": args.beta,
        "n_or": args.n_or,
        "link_format": args.prec,
        "link_updates_per_step_per_gpu": (1 + args.n_or) * 4 * V,
        "l2": "no flush: the link field (%.0f MB) is larger than the 129 MB L2" % (4 * V * LINK_BYTES[args.prec] / 1e6),
        "parallelism": "replicas",
    }


# ------------------------------------------------------------------ distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    def __init__(self, world, rank, local, use_cuda):
        self.world, self.rank, self.local = world, rank, local
        self.pg = None
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("nccl" if use_cuda else "gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch

        t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
# source files each profiled kernel is compiled from (shared headers + its .cu)
KERNEL_SOURCES = {
    "k_overrelax": "mgq_core.cu",
    "k_heatbath": "mgq_core.cu",
    "k_force": "mgq_hmc.cu",
}
_COMMON = ["mgq_device.cuh", "mgq_stencil.cuh", "mgq_internal.h"]


def src_hash(kernel: str) -> str:
    """Hash of the sources a kernel is compiled from; a profile summary whose
    hash differs was taken on other code."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1510_04675_gb300", "csrc")
    for f in _COMMON + [KERNEL_SOURCES[kernel]]:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel: str, workload_tag: str):
    """DRAM bytes per launch recorded by an ncu capture summary under profiles/,
    if it was taken on the current sources of that kernel."""
    if kernel not in KERNEL_SOURCES:
        return None
    cur = src_hash(kernel)
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.txt"))):
        for line in open(f):
            t = line.split()
            if len(t) >= 6 and t[0] == "traffic_bytes_per_launch" and t[1] == kernel and t[2] == workload_tag \
                    and t[4] == "src_hash":
                if t[5] == cur:
                    return float(t[3])
    return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(dims, beta, seconds_hint=20.0):
    """Time the FP64 oracle on one full compound sweep (1 HB + 4 OR) of a hot-start lattice."""
    import oracle

    oracle.build()
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    U = oracle.init_links(dims, 1, seed=7)
    V = U.shape[0]
    t0 = time.perf_counter()
    oracle.heatbath_sweep(U, dims, beta, 7, 0, 1, 1)
    for _ in range(4):
        oracle.overrelax_sweep(U, dims)
    dt = time.perf_counter() - t0
    return {"value": 5 * 4 * V / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one compound sweep (1 HB + 4 OR) of a hot-start {'x'.join(map(str, dims))} lattice, "
                      f"{5 * 4 * V} link updates in {dt:.2f} s (FP64, OpenMP)"}


def run_reference(args, dims, world, rank):
    """CPU oracle as the reference arm: each step is the mu = step mod 4 slice of a compound sweep."""
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    U = oracle.init_links(dims, 1, seed=7)
    V = U.shape[0]

    # one step: 1 HB + n_or OR updates of the links (mu = i mod 4, parity = (i//4) mod 2)
    # on one slab of L3/8 x3-planes (i//8 mod 8): V/16 sites per sub-sweep
    plane = dims[0] * dims[1] * dims[2]
    nslab = 8 if dims[3] % 8 == 0 else 1
    width = dims[3] // nslab

    def step(i):
        mu, par, slab = i % 4, (i // 4) % 2, (i // 8) % nslab
        lo, hi = slab * width * plane, (slab + 1) * width * plane
        oracle.subsweep_range(U, dims, 0, args.beta, 7, 0, i, 1, mu, par, lo, hi)
        for _ in range(args.n_or):
            oracle.subsweep_range(U, dims, 1, args.beta, 7, 0, i, 1, mu, par, lo, hi)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t0
    per_step = (1 + args.n_or) * (V // 2) // nslab
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, dims), link_format="f64 (oracle)",
                       sample="each step: one (mu, parity) subset of a compound sweep (1 HB + n_or OR) on one "
                              "x3-slab of 1/8 of the lattice"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps of {per_step} link updates each"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def ev():
    import torch

    return torch.cuda.Event(enable_timing=True)


def time_sweeps(api, lat, beta, n_or, steps, sweep0):
    """Link updates/s of `steps` compound sweeps (device-resident)."""
    import torch

    for i in range(2):
        api.mgq_update_sweeps(lat, beta, sweep0 + i, 1, 1, n_or)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    api.mgq_update_sweeps(lat, beta, sweep0 + 2, steps, 1, n_or)
    b.record()
    torch.cuda.synchronize()
    return (1 + n_or) * 4 * lat.volume * steps / (a.elapsed_time(b) * 1e-3)


def batched_leg(api, beta_lo=5.8, beta_hi=6.1, n_sweeps=20, n_or=4, seed=4242):
    """256 fine lattices (96 x 12^4, 96 x 16^4, 64 x 8^3x16, FP32 12-real) prolongated
    from coarse lattices thermalised at beta in [5.8, 6.1]; n_sweeps compound sweeps
    of all of them with per-lattice FP64 plaquettes, replayed from one CUDA graph."""
    import numpy as np
    import torch

    rng = np.random.default_rng(seed)
    shapes = [[12] * 4] * 96 + [[16] * 4] * 96 + [[8, 8, 8, 16]] * 64
    betas = rng.uniform(beta_lo, beta_hi, size=len(shapes)).tolist()
    coarse = [api.Lattice([d // 2 for d in s], "f32c12", seed=seed, lattice_id=i) for i, s in enumerate(shapes)]
    for c in coarse:
        api.mgq_init_links(c, 1)
    api.mgq_update_sweeps_batched(api.Batch(coarse, betas), 0, 30, 1, n_or)
    fine = [api.Lattice(s, "f32c12", seed=seed + 1, lattice_id=i) for i, s in enumerate(shapes)]
    for c, f in zip(coarse, fine):
        api.mgq_prolongate(c, f, 0.05, 0.0, 10)  # fixed 10 APE steps per stage
    del coarse
    batch = api.Batch(fine, betas, max_sweeps=1)
    P = batch.plaquette_buffer(1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for i in range(2):
            api.mgq_update_sweeps_batched(batch, i, 1, 1, n_or, P, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        api.mgq_update_sweeps_batched(batch, 2, 1, 1, n_or, P, stream=torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    for _ in range(n_sweeps):
        g.replay()
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) * 1e-3
    V = sum(int(np.prod(x)) for x in shapes)
    return {"lattices": len(shapes), "sites": V, "sweeps": n_sweeps,
            "link_updates_per_s": (1 + n_or) * 4 * V * n_sweeps / sec, "ms_per_sweep": 1e3 * sec / n_sweeps,
            "plaquette_mean": float(P.mean().item()), "graph": True,
            "workload": "96x12^4 + 96x16^4 + 64x8^3x16, beta in [5.8, 6.1], prolongated (10 APE steps/stage), "
                        "1 HB + 4 OR per sweep, FP32 12-real, per-lattice FP64 plaquette"}


def _timed(fn):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0


def hmc_leg(api, dims=(24, 24, 24, 24), beta=6.0, n_traj=100, n_warm=24, n_steps=20, prec="f32c12"):
    """HMC from a hot start: tau = 1, n_steps leapfrog steps, the first n_warm
    trajectories without accept/reject (Sec. IV.E)."""
    import numpy as np

    lat = api.Lattice(list(dims), prec, seed=2468, with_mom=True)
    api.mgq_init_links(lat, 1)
    api.mgq_hmc_trajectory(lat, beta, 1.0, n_steps, 10**6, 0)  # warm the code path
    api.mgq_init_links(lat, 1)
    out = []
    _, sec = _timed(lambda: [out.append(api.mgq_hmc_trajectory(lat, beta, 1.0, n_steps, t, 0 if t < n_warm else 1))
                             for t in range(n_traj)])
    dH = np.array([o[0] for o in out])
    acc = np.array([o[1] for o in out])
    return {"workload": f"{'x'.join(map(str, dims))} beta={beta} HMC, tau=1, {n_steps} steps, {n_traj} trajectories "
                        f"from a hot start ({n_warm} without accept/reject), {prec} links, FP64 H",
            "trajectories_per_s": n_traj / sec, "ms_per_trajectory": 1e3 * sec / n_traj,
            "acceptance_after_warmup": float(acc[n_warm:].mean()), "final_abs_dH": float(abs(dH[-1])),
            "plaquette": api.mgq_plaquette(lat)}


def multiscale_leg(api, beta_c=5.7, beta_f=6.0, n_sweeps=50, prec="f32c12"):
    """Multiscale step: coarse 8^4 (thermalised in-run) -> 16^4 prolongation with
    the paper's 0.001 % stopping rule, 50 rethermalisation sweeps, flow to t = 1."""
    c = api.Lattice([8, 8, 8, 8], prec, seed=1357)
    api.mgq_init_links(c, 1)
    api.mgq_update_sweeps(c, beta_c, 0, 100, 1, 4)
    f = api.Lattice([16, 16, 16, 16], prec, seed=1358)
    (iters, sd), t_pro = _timed(lambda: api.mgq_prolongate(c, f, 0.05, 1e-5, 10000))
    p_pro = api.mgq_plaquette(f)
    plaq, t_th = _timed(lambda: api.mgq_update_sweeps(f, beta_f, 0, n_sweeps, 1, 4, plaq_out=True))
    (E, Q), t_fl = _timed(lambda: api.mgq_wilson_flow(f, 0.01, 100, 100))
    return {"workload": "8^4 beta=5.7 -> 16^4 prolongation (c=0.05, 1e-5), 50 x (HB + 4 OR) at beta=6.0, "
                        f"Wilson flow eps=0.01 to t=1, clover E and Q; {prec} links, FP64 sums",
            "ape_iterations": iters, "ms_prolongation": 1e3 * t_pro, "ms_rethermalisation": 1e3 * t_th,
            "ms_flow": 1e3 * t_fl, "plaquette_prolongated": p_pro, "plaquette_after": float(plaq[-1]),
            "E_t1": float(E[-1]), "Q_t1": float(Q[-1])}


def flow_leg(api, dims=(24, 24, 24, 48), beta=5.96, t0=2.79, prec="f32c12"):
    """Wilson flow as in Sec. IV.B / Table II on the 24^3 x 48, beta = 5.96
    ensemble (nominal t0 = 2.79): adaptive step (tolerance 0.01, maximal step
    0.2, measurements every t0/4) to 14 t0, against the fixed step 0.01 to
    5 t0 on the same configuration."""
    import numpy as np

    lat = api.Lattice(list(dims), prec, seed=8642)
    api.mgq_init_links(lat, 1)
    api.mgq_update_sweeps(lat, beta, 0, 300, 1, 4)
    ref = api.copy_lattice(lat)
    n_fixed = int(round(5 * t0 / 0.01))
    (Ef, Qf), t_fix = _timed(lambda: api.mgq_wilson_flow(ref, 0.01, n_fixed, n_fixed // 5))
    (E, Q, steps, rejects), t_ad = _timed(lambda: api.mgq_wilson_flow_adaptive(lat, 14 * t0, 0.01, 0.2, 0.01, t0 / 4))
    Ea, Qa = E[0:21:4], Q[0:21:4]  # t = k t0, k = 0..5
    return {"workload": f"{'x'.join(map(str, dims))} beta={beta} (300 x (HB + 4 OR) from a hot start), {prec}; "
                        f"adaptive tol 0.01, max step 0.2, E/Q every t0/4 to 14 t0 vs fixed 0.01 to 5 t0",
            "adaptive_ms": 1e3 * t_ad, "adaptive_steps": steps, "adaptive_rejects": rejects,
            "fixed_ms": 1e3 * t_fix, "fixed_steps": n_fixed, "ms_per_fixed_step": 1e3 * t_fix / n_fixed,
            "max_rel_dev_E_to_5t0": float(np.max(np.abs(Ea - Ef) / Ef)),
            "max_abs_dev_Q_to_5t0": float(np.max(np.abs(Qa - Qf))), "Q_14t0": float(Q[-1]),
            "t2E_at_t0": float(t0 * t0 * Ea[1])}


def large_leg(api, beta=6.2):
    """48^4 at beta = 6.2, FP32 12-real and FP64 side by side: sweeps, HMC, flow to t = 3."""
    out = {}
    for prec, n_sw, n_traj, n_flow in [("f32c12", 100, 10, 300), ("f64", 2, 1, 10)]:
        lat = api.Lattice([48] * 4, prec, seed=97, with_mom=True)
        api.mgq_init_links(lat, 1)
        _, t_sw = _timed(lambda: api.mgq_update_sweeps(lat, beta, 0, n_sw, 1, 1))
        _, t_h = _timed(lambda: [api.mgq_hmc_trajectory(lat, beta, 1.0, 40, t, 0) for t in range(n_traj)])
        w = api.copy_lattice(lat)
        (E, Q), t_f = _timed(lambda: api.mgq_wilson_flow(w, 0.01, n_flow, n_flow))
        V = 48**4
        out[prec] = {"sweeps": n_sw, "link_updates_per_s": 2 * 4 * V * n_sw / t_sw,
                     "ms_per_hmc_trajectory_40_steps": 1e3 * t_h / n_traj, "ms_per_flow_step": 1e3 * t_f / n_flow,
                     "Q_flowed": float(Q[-1])}
        del w
        if prec == "f32c12":
            # dQ(W_t)/d omega at omega = 0 through the checkpointed adjoint flow (t = 3)
            import torch

            from paper_1510_04675_gb300.autograd import flowed_observable

            omega = torch.zeros_like(lat.new_alg_field(), requires_grad=True)

            def fwd_bwd():
                q = flowed_observable(omega, lat, "Q", 0.01, n_flow)
                q.backward()
                return q

            q, t_fb = _timed(fwd_bwd)
            out[prec]["ms_flowed_Q_forward_backward"] = 1e3 * t_fb
            out[prec]["grad_norm"] = float(omega.grad.norm())
            out[prec]["Q_flowed_autograd"] = float(q.detach())
            del omega
        del lat
    return out


def run_mgq(args, dims, world, rank, local):
    import torch

    from paper_1510_04675_gb300 import api
    from paper_1510_04675_gb300 import build as mgq_build

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for --impl mgq")
    torch.cuda.set_device(local)
    mgq_build.build()
    dist = Dist(world, rank, local, True)
    V = 1
    for d in dims:
        V *= d
    beta, n_or, K, W = args.beta, args.n_or, args.steps, args.warmup
    if n_or < 2:
        raise SystemExit("bench.py times plain and plaquette-measuring overrelaxation sweeps: needs --n-or >= 2")

    lat = api.Lattice(dims, args.prec, seed=1234, lattice_id=rank, with_mom=True)
    api.mgq_init_links(lat, 1)
    api.mgq_update_sweeps(lat, beta, 0, args.therm, 1, n_or)
    plaq_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    sweep0 = 1000

    hb_ev, or_ev, last_ev = [], [], []

    # one step: a heat-bath sweep, n_or overrelaxation sweeps, the plaquette;
    # the last overrelaxation sweep measures the plaquette as it goes
    def step(i, record):
        if record:
            e = (ev(), ev(), ev(), ev())
            e[0].record()
        api.mgq_heatbath_sweep(lat, beta, sweep0 + i, 1)
        if record:
            e[1].record()
        for _ in range(n_or - 1):
            api.mgq_overrelax_sweep(lat)
        if record:
            e[2].record()
        api.mgq_overrelax_sweep_plaquette(lat, out=plaq_dev)
        if record:
            e[3].record()
            hb_ev.append((e[0], e[1]))
            or_ev.append((e[1], e[2]))
            last_ev.append((e[2], e[3]))

    for i in range(W):
        step(i, False)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    t0, t1 = ev(), ev()
    t0.record()
    for i in range(K):
        step(W + i, True)
    t1.record()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_local = t0.elapsed_time(t1) * 1e-3
    t = dist.max(t_local)
    updates_per_step = (1 + n_or) * 4 * V
    value = world * K * updates_per_step / t

    # dominant kernel and its roofline (per-launch algorithmic bytes / average launch time)
    hb_ms = sum(a.elapsed_time(b) for a, b in hb_ev) / (8 * K)
    or_ms = sum(a.elapsed_time(b) for a, b in or_ev) / (8 * (n_or - 1) * K)
    last_ms = sum(a.elapsed_time(b) for a, b in last_ev) / K
    lb = LINK_BYTES[args.prec]
    bytes_per_launch = (V // 2) * 9 * lb  # 9 link transfers per link update, V/2 updates per launch
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"
    tag = "x".join(map(str, dims)) + "_" + args.prec
    kernels = {"k_heatbath": hb_ms, "k_overrelax": or_ms}
    share = {"k_heatbath": 8 * hb_ms, "k_overrelax": 8 * n_or * or_ms}
    dom = max(share, key=share.get)

    def roof(name, ms):
        ach = bytes_per_launch / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": traffic_from_profiles(name, tag), "kernel": name, "ms_per_launch": ms,
                "algorithmic_bytes_per_launch": bytes_per_launch, "peak_source": peak_src}

    def alu_roof(name, links, ms):
        if args.prec == "f64":
            return None
        ach = FLOPS_PER_LINK[name] * links / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS, "traffic": None, "kernel": name, "ms_per_launch": ms,
                "algorithmic_flops_per_link": FLOPS_PER_LINK[name], "peak_source": "derived (unit counts x clock)"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * t / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec != "f64" else "f64", "data": "synthetic (hot start, thermalised in-run)",
        "config": workload_config(args, dims),
        "roofline": roof(dom, kernels[dom]),
        "roofline_heatbath": roof("k_heatbath", hb_ms),
        "roofline_alu": {"k_overrelax": alu_roof("k_overrelax", V // 2, or_ms),
                         "k_heatbath": alu_roof("k_heatbath", V // 2, hb_ms)},
        "gpu_launches": K * (8 + 8 * n_or + 1),
        "ms_overrelax_sweep_with_plaquette": last_ms,
        "clocks": clocks,
    }

    # HMC force + momentum update (algorithmic GB/s: links once + P read and written)
    try:
        F = lat.new_alg_field()
        for _ in range(3):
            api.mgq_hmc_force(lat, beta, F)
        torch.cuda.synchronize()
        a, b = ev(), ev()
        nf = 20
        a.record()
        for _ in range(nf):
            api.mgq_hmc_force(lat, beta, F)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / nf
        fb = 4 * V * (lb + 8 * REAL_BYTES[args.prec])
        out["force_gbs"] = fb / (ms * 1e-3) / 1e9
        out["force_ms"] = ms
        out["force_roofline_frac"] = out["force_gbs"] / peak
        out["force_roofline"] = alu_roof("k_force", 4 * V, ms)
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        out["force_gbs"] = None
        out["force_error"] = str(e)[:200]

    # End to end through the C ABI: every step uploads its input links from pinned
    # host memory and reads its plaquette back to pinned host memory.  Two device
    # buffers let the upload of step i+1 (copy stream) overlap the sweeps of step i.
    host_links = lat.links.cpu().pin_memory()
    lat2 = api.copy_lattice(lat)
    bufs = (lat, lat2)
    ne = max(4, min(K, 20))
    ms, cs = torch.cuda.current_stream(), torch.cuda.Stream()
    plaq_dev = torch.zeros(ne, dtype=torch.float64, device="cuda")
    plaq_host = torch.zeros(ne, dtype=torch.float64).pin_memory()

    def e2e_run(sweep_base):
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        free = [None, None]
        for i in range(ne):
            b = i % 2
            with torch.cuda.stream(cs):
                if free[b] is not None:
                    cs.wait_event(free[b])
                bufs[b].links.copy_(host_links, non_blocking=True)
                ready[b].record(cs)
            ms.wait_event(ready[b])
            api.mgq_update_sweeps(bufs[b], beta, sweep_base + i, 1, 1, n_or, plaq_out=plaq_dev[i:i + 1])
            plaq_host[i:i + 1].copy_(plaq_dev[i:i + 1], non_blocking=True)
            free[b] = torch.cuda.Event()
            free[b].record(ms)
        ms.synchronize()

    e2e_run(sweep0 + 5000)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    e2e_run(sweep0 + 6000)
    we = time.perf_counter() - w0
    e2e_t = dist.max(we)
    out["e2e"] = {"value": world * ne * updates_per_step / e2e_t, "unit": UNIT,
                  "h2d_bytes_per_step": int(host_links.numel()), "d2h_bytes_per_step": 8,
                  "steps": ne, "plaquette_last": float(plaq_host[-1]),
                  "overlap": "double-buffered: the upload of step i+1 runs on a copy stream during step i"}
    del lat2

    if not args.no_extras and rank == 0:
        for prec, key in [("f64", "fp64_plain"), ("f32", "fp32_18real")]:
            l2 = api.Lattice(dims, prec, seed=99)
            api.mgq_init_links(l2, 1)
            api.mgq_update_sweeps(l2, beta, 0, 2, 1, n_or)
            r = time_sweeps(api, l2, beta, n_or, 2 if prec == "f64" else 5, 10)
            out[key + "_link_updates_per_s"] = r
            del l2
        out["speedup_vs_fp64"] = (value / world) / out["fp64_plain_link_updates_per_s"]
        del lat, host_links
        torch.cuda.empty_cache()
        legs = [("batched", batched_leg), ("hmc_24", hmc_leg), ("multiscale_16", multiscale_leg),
                ("flow_24x48", flow_leg)]
        if args.large:
            legs.append(("large_48", large_leg))
        for name, fn in legs:
            try:
                out[name] = fn(api)
            except Exception as e:  # noqa: BLE001 - reported in the line
                out[name] = {"error": str(e)[:200]}
            torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample(dims, beta)
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


def main():
    args = parse_args()
    dims = [int(v) for v in args.dims.split(",")]
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, dims, world, rank)
    return run_mgq(args, dims, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
