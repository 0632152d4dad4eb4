"""Multiscale thermalization workflow (Sec. II, IV) driven through the C ABI,
with metrics written as JSON lines.

  coarse lattice: hot start, heat bath + overrelaxation at beta_coarse
  -> prolongation to the doubled lattice (transfer + APE stages, Sec. III)
  -> rethermalisation at beta_fine (per-sweep plaquette, checkpoints)
  -> optional HMC trajectories (dH, acceptance; warm-up without the test)
  -> Wilson flow (fixed or adaptive step): E(t), Q(t), t0, chi

Every step runs in the library's kernels; this module only sequences calls
and records their results.  Run as
``python -m paper_1510_04675_gb300.driver --coarse 8 8 8 8 --log run.jsonl``.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from dataclasses import asdict, dataclass, field
from typing import IO, List, Optional

import numpy as np


@dataclass
class WorkflowConfig:
    coarse: List[int] = field(default_factory=lambda: [8, 8, 8, 8])
    beta_coarse: float = 5.7
    coarse_sweeps: int = 100
    beta_fine: float = 6.0
    retherm_sweeps: int = 50
    n_hb: int = 1
    n_or: int = 4
    prec: str = "f32c12"
    seed: int = 1
    ape_c: float = 0.05
    ape_tol: float = 1e-5
    hmc_trajectories: int = 0
    hmc_steps: int = 20
    hmc_warmup: int = 24
    flow: str = "adaptive"  # "none", "fixed" or "adaptive"
    flow_t: float = 1.0
    flow_eps: float = 0.01  # fixed step, or the first trial step of the adaptive flow
    flow_tol: float = 0.01
    flow_max_step: float = 0.2
    flow_dt_meas: float = 0.25
    checkpoint_every: int = 0
    checkpoint_dir: Optional[str] = None


class JsonlLog:
    """One JSON object per line: {"kind": ..., "wall_s": ..., **fields}."""

    def __init__(self, stream: Optional[IO[str]] = None):
        self.stream = stream
        self.t0 = time.perf_counter()
        self.records: List[dict] = []

    def write(self, kind: str, **fields) -> None:
        rec = {"kind": kind, "wall_s": round(time.perf_counter() - self.t0, 6), **fields}
        self.records.append(rec)
        if self.stream is not None:
            self.stream.write(json.dumps(rec) + "\n")
            self.stream.flush()


def run(cfg: WorkflowConfig, log: JsonlLog) -> dict:
    import torch

    from . import api
    from .analysis import susceptibility, t0_from_flow

    log.write("config", **asdict(cfg))
    c = api.Lattice(cfg.coarse, cfg.prec, seed=cfg.seed, lattice_id=0)
    api.mgq_init_links(c, 1)
    plaq = api.mgq_update_sweeps(c, cfg.beta_coarse, 0, cfg.coarse_sweeps, cfg.n_hb, cfg.n_or, plaq_out=True)
    for i, p in enumerate(plaq):
        log.write("coarse_sweep", sweep=i, plaquette=float(p))

    fine_dims = [2 * d for d in cfg.coarse]
    f = api.Lattice(fine_dims, cfg.prec, seed=cfg.seed, lattice_id=1, with_mom=cfg.hmc_trajectories > 0)
    iters, sd = api.mgq_prolongate(c, f, cfg.ape_c, cfg.ape_tol)
    log.write("prolongation", dims=fine_dims, ape_iterations=iters, partial_actions=sd,
              plaquette=api.mgq_plaquette(f))
    del c

    done = 0
    chunk = cfg.checkpoint_every if cfg.checkpoint_every > 0 else cfg.retherm_sweeps
    while done < cfg.retherm_sweeps:
        n = min(chunk, cfg.retherm_sweeps - done, 500)
        plaq = api.mgq_update_sweeps(f, cfg.beta_fine, done, n, cfg.n_hb, cfg.n_or, plaq_out=True)
        for i, p in enumerate(plaq):
            log.write("sweep", sweep=done + i, plaquette=float(p))
        done += n
        if cfg.checkpoint_every > 0 and cfg.checkpoint_dir:
            os.makedirs(cfg.checkpoint_dir, exist_ok=True)
            path = os.path.join(cfg.checkpoint_dir, f"fine_{done:06d}.mgq")
            api.save_checkpoint(f, path, cfg.beta_fine, done)
            log.write("checkpoint", sweep=done, path=path)

    acc = []
    for traj in range(cfg.hmc_trajectories):
        test = 1 if traj >= cfg.hmc_warmup else 0
        dH, a = api.mgq_hmc_trajectory(f, cfg.beta_fine, 1.0, cfg.hmc_steps, traj, test)
        if test:
            acc.append(a)
        log.write("hmc", trajectory=traj, dH=dH, accepted=a, metropolis=bool(test), plaquette=api.mgq_plaquette(f))

    summary = {"plaquette": api.mgq_plaquette(f), "sweeps": done,
               "hmc_acceptance": float(np.mean(acc)) if acc else None}
    if cfg.flow != "none":
        w = api.copy_lattice(f)
        if cfg.flow == "fixed":
            n_steps = int(round(cfg.flow_t / cfg.flow_eps))
            every = max(1, int(round(cfg.flow_dt_meas / cfg.flow_eps)))
            E, Q = api.mgq_wilson_flow(w, cfg.flow_eps, n_steps, every)
            t = cfg.flow_eps * every * np.arange(len(E))
            extra = {}
        elif cfg.flow == "adaptive":
            E, Q, steps, rejects = api.mgq_wilson_flow_adaptive(w, cfg.flow_t, cfg.flow_tol, cfg.flow_max_step,
                                                                cfg.flow_eps, cfg.flow_dt_meas)
            t = np.minimum(cfg.flow_dt_meas * np.arange(len(E)), cfg.flow_t)
            extra = {"steps": steps, "rejects": rejects}
        else:
            raise ValueError(f"unknown flow mode {cfg.flow!r}")
        for ti, e, q in zip(t, E, Q):
            log.write("flow", t=float(ti), E=float(e), t2E=float(ti * ti * e), Q=float(q))
        V = int(np.prod(fine_dims))
        summary.update({"t0": t0_from_flow(t, E), "Q": float(Q[-1]), "chi": susceptibility([Q[-1]], V), **extra})
        del w
    torch.cuda.synchronize()
    log.write("summary", **summary)
    return summary


def main(argv=None) -> int:
    d = WorkflowConfig()
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--coarse", type=int, nargs=4, default=d.coarse)
    for name in ("beta_coarse", "beta_fine", "ape_c", "ape_tol", "flow_t", "flow_eps", "flow_tol", "flow_max_step",
                 "flow_dt_meas"):
        ap.add_argument("--" + name.replace("_", "-"), type=float, default=getattr(d, name))
    for name in ("coarse_sweeps", "retherm_sweeps", "n_hb", "n_or", "seed", "hmc_trajectories", "hmc_steps",
                 "hmc_warmup", "checkpoint_every"):
        ap.add_argument("--" + name.replace("_", "-"), type=int, default=getattr(d, name))
    ap.add_argument("--prec", choices=["f64", "f32", "f32c12"], default=d.prec)
    ap.add_argument("--flow", choices=["none", "fixed", "adaptive"], default=d.flow)
    ap.add_argument("--checkpoint-dir", default=None)
    ap.add_argument("--log", default="-", help="JSONL output path ('-' = stdout)")
    a = ap.parse_args(argv)
    cfg = WorkflowConfig(**{k: getattr(a, k) for k in asdict(d)})
    out = sys.stdout if a.log == "-" else open(a.log, "w")
    try:
        run(cfg, JsonlLog(out))
    finally:
        if out is not sys.stdout:
            out.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
