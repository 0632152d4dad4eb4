"""Host analysis helpers and the workflow driver's logging (no GPU)."""
import io
import json

import numpy as np
import pytest

from paper_1510_04675_gb300.analysis import susceptibility, t0_from_flow
from paper_1510_04675_gb300.driver import JsonlLog, WorkflowConfig, main


def test_t0_linear_interpolation_is_exact_on_a_linear_curve():
    # t^2 E(t) = 0.2 + 0.1 t  ->  t0 = 1 exactly, measurements do not hit it
    t = np.array([0.0, 0.3, 0.7, 1.4, 2.0])
    E = np.zeros_like(t)
    E[1:] = (0.2 + 0.1 * t[1:]) / t[1:] ** 2
    assert t0_from_flow(t, E) == pytest.approx(1.0, rel=1e-14)


def test_t0_brackets_and_edge_cases():
    t = np.array([0.0, 1.0, 2.0])
    E = np.array([0.0, 0.1, 0.1])  # t^2 E = 0, 0.1, 0.4 -> crossing at 1 + 0.2/0.3
    assert t0_from_flow(t, E) == pytest.approx(1 + 2 / 3)
    assert np.isnan(t0_from_flow(t, np.array([0.0, 0.01, 0.01])))
    with pytest.raises(ValueError):
        t0_from_flow(t, E[:2])


def test_susceptibility():
    assert susceptibility([2.0, -2.0, 0.0], 8) == pytest.approx(8 / 3 / 8)
    with pytest.raises(ValueError):
        susceptibility([], 8)


def test_jsonl_log_records_and_cli_rejects_bad_flags():
    buf = io.StringIO()
    log = JsonlLog(buf)
    log.write("sweep", sweep=3, plaquette=0.5)
    rec = json.loads(buf.getvalue())
    assert rec["kind"] == "sweep" and rec["sweep"] == 3 and rec["plaquette"] == 0.5 and rec["wall_s"] >= 0
    assert WorkflowConfig().coarse == [8, 8, 8, 8]
    with pytest.raises(SystemExit):
        main(["--flow", "sideways"])


def test_tau_int_of_an_ar1_process():
    """The windowed integrated autocorrelation time used by the chain
    comparisons: an AR(1) process x_t = r x_{t-1} + e_t has tau_int =
    (1 + r) / (2 (1 - r))."""
    from test_gpu_update import _tau_int

    rng = np.random.default_rng(5)
    for r in (0.0, 0.5, 0.8):
        x = np.zeros(40000)
        e = rng.standard_normal(x.size)
        for t in range(1, x.size):
            x[t] = r * x[t - 1] + e[t]
        want = (1 + r) / (2 * (1 - r))
        assert abs(_tau_int(x) - want) < 0.12 * want + 0.05, (r, _tau_int(x), want)
