"""Estimators read off the int64 accumulators (paper_1004_0023_gb300/estimators.py), checked
on oracle runs against exact results: exact diagonalisation for the quantum energy, the
transfer-matrix moments for E and M, and the counters for the rates."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import estimators, instances
from tests import exact


def test_moments_and_quantum_energy_match_exact_results():
    prob = instances.tiny_problem(3, [(0, 1), (1, 2)], [1, -1], [1, 0, -1], 32, [1.0], [1.0], seed=21)
    ed = exact.exact_diag(prob, 0)
    tm = exact.transfer_matrix(prob, 0)
    trotter = abs(exact.st_energy_estimator(tm["E"], tm["M"], 3, 32, 1.0, 1.0) - ed)
    o = Oracle.from_problem(prob)
    o.run(2000, 1)  # burn-in, excluded with `since`
    start = o.obs()
    rows_h, rows_e, rows_m = [], [], []
    prev = start
    for _ in range(30):
        o.run(2500, 1)
        cur = o.obs()
        rows_h.append(estimators.quantum_energy(cur, 3, 32, prob.T, prob.gamma, since=prev)[0])
        m = estimators.moments(cur, since=prev)
        rows_e.append(m["E"][0])
        rows_m.append(m["M"][0])
        prev = cur
    for rows, want, extra in ((rows_h, ed, trotter), (rows_e, tm["E"], 0.0), (rows_m, tm["M"], 0.0)):
        rows = np.asarray(rows)
        se = rows.std(ddof=1) / np.sqrt(rows.size)
        assert abs(rows.mean() - want) < 5 * se + extra, (rows.mean(), want, se)
    # the whole window equals the mean of the sub-windows (same number of sweeps each)
    whole = estimators.moments(prev, since=start)
    assert np.isclose(whole["E"][0], np.mean(rows_e)) and whole["n"][0] == 30 * 2500


def test_rates_follow_the_counters():
    prob = instances.workload("regular3_n16_p32_r16", 3)
    o = Oracle.from_problem(prob)
    o.run(300, 1)
    ob = o.obs()
    fr = estimators.flip_rate(ob, prob.n, prob.P)
    assert np.allclose(fr, np.asarray(ob["flip_acc"]) / (300 * prob.n * prob.P))
    assert np.all((fr >= 0) & (fr <= 1))
    sr = estimators.swap_rate(ob)
    assert sr.shape == (prob.R - 1,) and np.all((sr >= 0) & (sr <= 1))
    assert np.allclose(sr, np.asarray(ob["swap_acc"]) / np.maximum(np.asarray(ob["swap_att"]), 1))
    # the high-Gamma end of the ladder flips more often than the low end at T = 0.05
    assert fr[-1] > fr[0]


def test_round_trips_on_hand_made_histories():
    # two rungs, chains alternating: each completes one bottom -> top -> bottom trip
    assert estimators.round_trips([[0, 1], [1, 0], [0, 1], [1, 0], [1, 0]]).tolist() == [1, 1]
    # three rungs (replica_at[r] = chain on rung r), traced by hand: chain 2 reaches the
    # bottom at steps 0, 3, 6 and 8 with a top visit in between each time (3 trips); chain 1
    # is at the bottom at step 1 and the top at step 3, back at the bottom at step 5 (1 trip);
    # chain 0 first reaches the bottom at step 4 and never returns
    hist = [[2, 1, 0], [1, 2, 0], [1, 0, 2], [2, 0, 1], [0, 1, 2], [1, 2, 0], [2, 1, 0], [1, 0, 2], [2, 1, 0]]
    assert estimators.round_trips(hist).tolist() == [0, 1, 3]
    assert estimators.round_trips([]).size == 0


# ---------------------------------------------------------------------------------------
# Batch means, error bars and integrated autocorrelation times. The estimator only sees the
# accumulators (count, sum, sum of squares) read at window boundaries; these pins feed it
# series whose autocorrelation time has a closed form, through that same interface.

def _history_from_series(x, y, window):
    """Observation dicts read every `window` samples of two integer series (as E and M)."""
    x = np.asarray(x, np.int64)
    y = np.asarray(y, np.int64)
    nb = x.size // window
    hist = []
    zeros = np.zeros(1, np.int64)
    for b in range(nb + 1):
        m = b * window
        hist.append({"n_meas": np.array([m]), "sum_E": np.array([x[:m].sum()]), "sum_E2": np.array([(x[:m] ** 2).sum()]),
                     "sum_M": np.array([y[:m].sum()]), "sum_M2": np.array([(y[:m] ** 2).sum()]),
                     "flip_acc": zeros, "swap_att": zeros, "swap_acc": zeros})
    return hist


def _two_state_chain(p, n, rng):
    """+-1 Markov chain that flips with probability p each step: rho(t) = (1 - 2p)^t,
    so tau = 1/2 + sum_t rho(t) = (1 - p) / (2 p)."""
    flips = rng.random(n) < p
    return np.where(np.cumsum(flips) % 2 == 0, 1, -1)


def _ar1(rho, n, rng, scale=10000):
    """AR(1) x_t = rho x_{t-1} + sqrt(1 - rho^2) e_t from a stationary start, scaled to
    integers: rho(t) = rho^t, so tau = (1 + rho) / (2 (1 - rho))."""
    signal = pytest.importorskip("scipy.signal")
    e = rng.standard_normal(n) * np.sqrt(1 - rho * rho)
    x0 = rng.standard_normal()
    x, _ = signal.lfilter([1.0], [1.0, -rho], e, zi=[rho * x0])
    return np.rint(scale * x).astype(np.int64)


def test_autocorrelation_time_of_a_two_state_chain_and_iid_samples():
    rng = np.random.default_rng(7)
    n, window = 1 << 21, 2048
    p_e, p_m = 0.05, 0.2
    x = _two_state_chain(p_e, n, rng)
    y = rng.choice([-1, 1], size=n)  # iid: tau = 1/2
    res = estimators.autocorrelation(_history_from_series(x, y, window))
    tau_e = (1 - p_e) / (2 * p_e)
    assert abs(res["E"]["tau"][0] / tau_e - 1) < 0.15, (res["E"]["tau"], tau_e)
    assert abs(res["M"]["tau"][0] / 0.5 - 1) < 0.15, res["M"]["tau"]
    # the error of the mean is sqrt(2 tau var / n); the effective sample size n / (2 tau)
    assert abs(res["E"]["err"][0] / np.sqrt(2 * tau_e * 1.0 / n) - 1) < 0.15
    assert abs(res["E"]["ess"][0] / (n / (2 * tau_e)) - 1) < 0.15
    assert abs(res["M"]["ess"][0] / n - 1) < 0.15
    # a second two-state chain with a short time
    z = _two_state_chain(p_m, n, rng)
    res2 = estimators.autocorrelation(_history_from_series(z, y, window))
    assert abs(res2["E"]["tau"][0] / ((1 - p_m) / (2 * p_m)) - 1) < 0.15


def test_autocorrelation_time_of_an_ar1_series():
    rng = np.random.default_rng(11)
    n, window, rho = 1 << 20, 2048, 0.8
    x = _ar1(rho, n, rng)
    res = estimators.autocorrelation(_history_from_series(x, x, window))
    tau = (1 + rho) / (2 * (1 - rho))
    assert abs(res["E"]["tau"][0] / tau - 1) < 0.15, (res["E"]["tau"], tau)
    assert abs(res["E"]["mean"][0] / 10000.0) < 5 * np.sqrt(2 * tau / n) + 1e-3


def test_batch_means_errors_match_the_spread_over_independent_seeds():
    # the same small problem under 12 independent Philox seeds: the batch-means error of
    # one run predicts the spread of the run means across seeds
    means_e, errs_e, means_h, errs_h = [], [], [], []
    for seed in range(12):
        prob = instances.tiny_problem(3, [(0, 1), (1, 2)], [1, -1], [1, 0, -1], 16, [1.0, 0.7], [1.0, 1.2],
                                      seed=1000 + seed)
        o = Oracle.from_problem(prob)
        o.run(500, 1)
        hist = [o.obs()]
        for _ in range(32):
            o.run(400, 1)
            hist.append(o.obs())
        o.close()
        res = estimators.autocorrelation(hist, 3, 16, prob.T, prob.gamma)
        means_e.append(res["E"]["mean"])
        errs_e.append(res["E"]["err"])
        means_h.append(res["H"]["mean"])
        errs_h.append(res["H"]["err"])
        assert np.all(res["E"]["tau"] > 0.4)
    for means, errs in ((means_e, errs_e), (means_h, errs_h)):
        spread = np.std(np.asarray(means), axis=0, ddof=1)
        ratio = np.mean(np.asarray(errs), axis=0) / spread
        assert np.all((ratio > 0.55) & (ratio < 1.8)), ratio


def test_rate_errors_and_window_sums_are_exact_differences():
    prob = instances.workload("regular3_n16_p32_r16", 2)
    o = Oracle.from_problem(prob)
    hist = [o.obs()]
    for _ in range(5):
        o.run(40, 1)
        hist.append(o.obs())
    o.close()
    w = estimators.window_sums(hist)
    assert w["n_meas"].shape == (5, prob.R) and np.all(w["n_meas"] == 40)
    assert np.array_equal(w["sum_E"].sum(axis=0), np.asarray(hist[-1]["sum_E"]) - np.asarray(hist[0]["sum_E"]))
    assert np.all(w["swap_att"] == 20)  # pairs of one parity per pass, alternating
    re = estimators.rate_errors(hist)
    assert re["flip_err"].shape == (prob.R,) and re["swap_err"].shape == (prob.R - 1,)
    assert np.all(re["flip_err"] >= 0)
