"""Physical estimators from the int64 accumulators a run leaves behind (host side).

The sweep kernels gather, after every sweep and per rung, the count n and the sums of E,
E^2, M and M^2 (the paper's "gather statistics" step of Fig. 4, accumulated in high
precision as in Sec. 5), plus accepted flips per rung and swap attempts / accepts per pair.
This module turns those into the quantities one reads off a PT-QMC run. It only reads
observables (the dict that `PT.obs()` or `Batch.obs()` returns, or two of them to take the
difference over a window) and does no sampling itself.

Suzuki-Trotter quantities at rung r (inverse temperature beta, field Gamma, P copies):
a = beta Gamma / P. With Z_P = (sinh(2a)/2)^(NP/2) sum_X exp(-S) and
S = (beta/P) E - K M, K = -1/2 ln tanh a, the thermal energy of the transverse-field
Hamiltonian is -d ln Z_P / d beta:
    <H> ~= <E>/P - N Gamma coth(2a) + Gamma <M> / (P sinh(2a)),
exact up to the O(1/P^2) Trotter error.
"""
from __future__ import annotations

import numpy as np


def _window(obs, since=None):
    """Per-rung sums over the sweeps between `since` (an earlier obs dict) and `obs`."""
    keys = ("n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc", "swap_att", "swap_acc")
    cur = {k: np.asarray(obs[k], np.float64) for k in keys}
    if since is not None:
        for k in keys:
            cur[k] = cur[k] - np.asarray(since[k], np.float64)
    return cur


def moments(obs, since=None):
    """Per-rung means and variances of E (summed over copies) and of the Trotter sum M."""
    w = _window(obs, since)
    n = np.maximum(w["n_meas"], 1.0)
    mE, mM = w["sum_E"] / n, w["sum_M"] / n
    return {"n": w["n_meas"], "E": mE, "M": mM,
            "var_E": np.maximum(w["sum_E2"] / n - mE * mE, 0.0),
            "var_M": np.maximum(w["sum_M2"] / n - mM * mM, 0.0)}


def quantum_energy(obs, N, P, T, gamma, since=None):
    """Thermal <H> per rung from the ST moments (formula in the module docstring)."""
    m = moments(obs, since)
    beta = 1.0 / np.asarray(T, np.float64)
    g = np.asarray(gamma, np.float64)
    a = beta * g / P
    return m["E"] / P - N * g / np.tanh(2.0 * a) + g * m["M"] / (P * np.sinh(2.0 * a))


def classical_energy(obs, P, since=None):
    """Mean problem energy of one Trotter copy per rung, <E>/P."""
    return moments(obs, since)["E"] / P


def flip_rate(obs, N, P, since=None):
    """Fraction of accepted Metropolis flips per rung (attempts = N P per sweep)."""
    w = _window(obs, since)
    return w["flip_acc"] / np.maximum(w["n_meas"] * N * P, 1.0)


def swap_rate(obs, since=None):
    """Accepted fraction of the swap attempts between rungs r and r + 1."""
    w = _window(obs, since)
    return w["swap_acc"] / np.maximum(w["swap_att"], 1.0)


def round_trips(replica_at_history):
    """Complete bottom-top-bottom trips of each chain through the ladder.

    replica_at_history: sequence of `replica_at` arrays (slot of the chain on each rung),
    one per observation, in time order. Each chain's trips are counted from its first visit
    to the bottom rung: a visit to the top rung then a return to the bottom rung makes one.
    """
    hist = [np.asarray(h) for h in replica_at_history]
    if not hist:
        return np.zeros(0, np.int64)
    R = hist[0].size
    trips = np.zeros(R, np.int64)
    state = np.zeros(R, np.int8)  # 0: not yet at the bottom, 1: bottom seen, 2: top seen after
    for h in hist:
        bottom, top = int(h[0]), int(h[R - 1])
        for chain in range(R):
            if chain == bottom:
                if state[chain] == 2:
                    trips[chain] += 1
                state[chain] = 1
            elif chain == top and state[chain] == 1:
                state[chain] = 2
    return trips
