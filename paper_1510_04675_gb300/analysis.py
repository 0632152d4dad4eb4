"""Scalar analysis of flow measurements (host arithmetic on values the
kernels returned): the reference scale t0 and the topological susceptibility.

t0 (Sec. IV.B): the flow time where t^2 E(t) = 0.3, found by linear
interpolation between the two neighbouring measurements of t^2 E(t).
chi (Sec. IV.C): <Q^2> / V.
"""
from __future__ import annotations

import numpy as np


def t0_from_flow(t, E, target: float = 0.3) -> float:
    """First crossing of t^2 E(t) = target, linearly interpolated between the
    two measurements that bracket it; NaN when the curve never reaches it."""
    t = np.asarray(t, dtype=np.float64)
    y = t * t * np.asarray(E, dtype=np.float64)
    if t.shape != y.shape or t.ndim != 1:
        raise ValueError("t and E must be 1-D arrays of the same length")
    above = np.nonzero(y >= target)[0]
    if above.size == 0:
        return float("nan")
    i = int(above[0])
    if i == 0:
        return float(t[0])
    t_lo, t_hi, y_lo, y_hi = t[i - 1], t[i], y[i - 1], y[i]
    return float(t_lo + (target - y_lo) * (t_hi - t_lo) / (y_hi - y_lo))


def susceptibility(Q, volume: int) -> float:
    """chi = <Q^2> / V over the configurations in Q."""
    Q = np.asarray(Q, dtype=np.float64)
    if Q.size == 0 or volume <= 0:
        raise ValueError("need at least one charge and a positive volume")
    return float(np.mean(Q * Q) / volume)
