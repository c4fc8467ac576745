"""Ladder adaptation for parallel tempering (host side).

The paper takes its ladder of (T, Gamma) rungs as given, generated beforehand by the method
of its ref. [7] (Sec. 2). This module offers the common feedback alternative: run, read the
swap acceptance rate A_r between rungs r and r + 1 (`estimators.swap_rate`), and move the
interior rungs so that every neighbouring pair accepts about equally often, which removes
the bottlenecks that stop chains from travelling along the ladder.

The rule: a pair with acceptance A behaves like a distance d = -ln A between its rungs.
The new rungs are placed at equal steps of cumulative distance, interpolating the rung
parameter (Gamma, or T for a classical ladder) piecewise linearly between the old rungs.
The two end rungs stay fixed and the ladder stays strictly monotone. Repeated runs with
`adapt` converge when all A_r are equal: a ladder with equal acceptance everywhere is a
fixed point.
"""
from __future__ import annotations

import numpy as np


def adapt(values, swap_acceptance, floor=1e-3):
    """New rung parameters (same length, same ends) from the current ones and the measured
    acceptance of each neighbouring pair (length len(values) - 1)."""
    x = np.asarray(values, np.float64)
    a = np.asarray(swap_acceptance, np.float64)
    if x.ndim != 1 or a.shape != (max(x.size - 1, 0),):
        raise ValueError("need R rung values and R - 1 pair acceptances")
    if x.size < 3:
        return x.copy()
    if not (np.all(np.diff(x) > 0) or np.all(np.diff(x) < 0)):
        raise ValueError("rung values must be strictly monotone")
    d = -np.log(np.clip(a, floor, 1.0))
    d = np.maximum(d, 1e-12)  # pairs that always swap still occupy some distance
    cum = np.concatenate([[0.0], np.cumsum(d)])
    targets = np.linspace(0.0, cum[-1], x.size)
    out = np.interp(targets, cum, x)
    out[0], out[-1] = x[0], x[-1]
    return out


def adapt_problem(prob, obs, since=None, floor=1e-3):
    """A copy of `prob` (an instances.Problem) with its ladder adapted from the swap rates
    in `obs` (optionally over the window since an earlier read). Gamma ladders move Gamma
    at fixed T; classical ladders (P = 1, Gamma = 0) move T."""
    import dataclasses

    from paper_1004_0023_gb300 import estimators

    rates = estimators.swap_rate(obs, since)
    if prob.P == 1:
        return dataclasses.replace(prob, T=adapt(prob.T, rates, floor))
    return dataclasses.replace(prob, gamma=adapt(prob.gamma, rates, floor))
