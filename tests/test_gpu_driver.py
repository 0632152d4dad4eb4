"""The multiscale workflow driver end to end on a small lattice: every stage
logs its records, checkpoints reload bit for bit, and the logged values are
the library's (prolongated plaquette, per-sweep plaquettes, flow)."""
import io
import json

import numpy as np
import pytest
import torch

from paper_1510_04675_gb300.driver import JsonlLog, WorkflowConfig, run

pytestmark = pytest.mark.gpu


def test_workflow_records(gpu, tmp_path):
    cfg = WorkflowConfig(coarse=[4, 4, 4, 4], coarse_sweeps=20, retherm_sweeps=10, hmc_trajectories=3,
                         hmc_warmup=2, hmc_steps=10, flow="adaptive", flow_t=0.6, flow_dt_meas=0.25,
                         checkpoint_every=5, checkpoint_dir=str(tmp_path))
    buf = io.StringIO()
    summary = run(cfg, JsonlLog(buf))
    recs = [json.loads(line) for line in buf.getvalue().splitlines()]
    kinds = [r["kind"] for r in recs]
    assert kinds.count("coarse_sweep") == 20 and kinds.count("sweep") == 10 and kinds.count("hmc") == 3
    assert kinds.count("checkpoint") == 2 and kinds.count("flow") == 4 and kinds[-1] == "summary"
    pro = next(r for r in recs if r["kind"] == "prolongation")
    assert pro["dims"] == [8, 8, 8, 8] and all(i >= 1 for i in pro["ape_iterations"])
    sweeps = [r["plaquette"] for r in recs if r["kind"] == "sweep"]
    assert all(0.0 < p < 1.0 for p in sweeps)
    hmc = [r for r in recs if r["kind"] == "hmc"]
    assert [h["metropolis"] for h in hmc] == [False, False, True]
    flow = [r for r in recs if r["kind"] == "flow"]
    assert [f["t"] for f in flow] == [0.0, 0.25, 0.5, 0.6]
    assert flow[-1]["E"] < flow[0]["E"]
    assert summary["steps"] >= 3 and np.isfinite(summary["Q"])
    # the second checkpoint holds the field after 10 rethermalisation sweeps
    last = [r for r in recs if r["kind"] == "checkpoint"][-1]
    lat, beta, sweep = gpu.load_checkpoint(last["path"])
    assert (beta, sweep) == (6.0, 10)
    # the record comes from the plaquette-measuring overrelaxation sweep:
    # the same field, summed differently (FP32 rounding of Re Tr U A)
    assert abs(gpu.mgq_plaquette(lat) - sweeps[-1]) < 1e-7
