"""Physical estimators from the int64 accumulators a run leaves behind (host side).

The sweep kernels gather, after every sweep and per rung, the count n and the sums of E,
E^2, M and M^2 (the paper's "gather statistics" step of Fig. 4, accumulated in high
precision as in Sec. 5), plus accepted flips per rung and swap attempts / accepts per pair.
This module turns those into the quantities one reads off a PT-QMC run. It only reads
observables (the dict that `PT.obs()` or `Batch.obs()` returns, two of them to take the
difference over a window, or a sequence of them read every W sweeps for batch means,
error bars and autocorrelation times) and does no sampling itself.

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


def window_sums(history):
    """Per-window sums between successive observations.

    history: observation dicts (as `PT.obs()` returns) read at successive times of one run,
    in time order. Returns a dict of arrays shaped [windows, R] (per pair for the swap
    counters): n_meas, sum_E, sum_E2, sum_M, sum_M2, flip_acc, swap_att, swap_acc, each the
    difference of the int64 accumulators between consecutive observations (exact integers).
    """
    keys = ("n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc", "swap_att", "swap_acc")
    if len(history) < 2:
        raise ValueError("need at least two observations")
    out = {}
    for k in keys:
        a = np.stack([np.asarray(h[k], np.int64) for h in history])
        out[k] = np.diff(a, axis=0)
    return out


def _batch_stats(wmean, n_per_window, var_sample):
    """Batch-means error, integrated autocorrelation time and effective sample size from the
    window means wmean[b, r] of windows of n_per_window[b, r] samples each.

    For a stationary series with variance s^2 and integrated autocorrelation time
    tau = 1/2 + sum_{t >= 1} rho(t), the mean of B consecutive samples has variance
    2 tau s^2 / B once B >> tau. So tau = B var(window means) / (2 s^2), the error of the
    overall mean is sqrt(var(window means) / windows), and the effective sample size is
    n / (2 tau). s^2 is the variance of the individual samples over the whole range.
    """
    nb = wmean.shape[0]
    if nb < 2:
        raise ValueError("need at least two windows")
    B = n_per_window.mean(axis=0)
    vb = wmean.var(axis=0, ddof=1)
    err = np.sqrt(vb / nb)
    tau = np.where(var_sample > 0, B * vb / (2.0 * np.maximum(var_sample, 1e-300)), np.nan)
    n_total = n_per_window.sum(axis=0)
    ess = np.where(tau > 0, n_total / (2.0 * np.where(tau > 0, tau, 1.0)), np.nan)
    return err, tau, ess


def autocorrelation(history, N=None, P=None, T=None, gamma=None):
    """Batch means over the windows between successive observations of one run (Fig. 4's
    statistics, read every W sweeps): per rung, for E and M (and for the quantum energy
    estimator when N, P, T and gamma are given), the mean over all windows, its standard
    error, the integrated autocorrelation time in sweeps and the effective sample size.
    Windows should be equally long and much longer than the autocorrelation time; the
    estimate of tau is then unbiased up to O(tau / window) and its relative error is about
    sqrt(2 / windows).
    """
    w = window_sums(history)
    n = w["n_meas"].astype(np.float64)
    if np.any(n <= 0):
        raise ValueError("every window needs at least one sweep")
    out = {"windows": int(n.shape[0]), "sweeps_per_window": n.mean(axis=0)}
    ntot = n.sum(axis=0)
    means = {}
    for key in ("E", "M"):
        s1 = w["sum_" + key].astype(np.float64)
        s2 = w["sum_" + key + "2"].astype(np.float64)
        wmean = s1 / n
        mean = s1.sum(axis=0) / ntot
        var_sample = np.maximum(s2.sum(axis=0) / ntot - mean * mean, 0.0)
        err, tau, ess = _batch_stats(wmean, n, var_sample)
        out[key] = {"mean": mean, "err": err, "tau": tau, "ess": ess}
        means[key] = wmean
    if N is not None and P is not None and T is not None and gamma is not None:
        beta = 1.0 / np.asarray(T, np.float64)
        g = np.asarray(gamma, np.float64)
        a = beta * g / P
        ce, cm = 1.0 / P, g / (P * np.sinh(2.0 * a))
        h_w = ce * means["E"] + cm * means["M"] - N * g / np.tanh(2.0 * a)
        # the per-sample variance of the linear combination needs cov(E, M), which the
        # accumulators do not hold; the error comes from the window means alone
        nb = h_w.shape[0]
        out["H"] = {"mean": (h_w * n).sum(axis=0) / ntot, "err": np.sqrt(h_w.var(axis=0, ddof=1) / nb)}
    return out


def rate_errors(history):
    """Batch-means errors of the flip rate per rung and the swap acceptance per pair."""
    w = window_sums(history)
    nb = w["n_meas"].shape[0]
    fr = w["flip_acc"] / np.maximum(w["n_meas"], 1)
    sr = w["swap_acc"] / np.maximum(w["swap_att"], 1)
    return {"flip_err": fr.std(axis=0, ddof=1) / np.sqrt(nb) if nb > 1 else np.full(fr.shape[1:], np.nan),
            "swap_err": sr.std(axis=0, ddof=1) / np.sqrt(nb) if nb > 1 else np.full(sr.shape[1:], np.nan)}


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
