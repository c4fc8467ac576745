"""Estimators read off the int64 accumulators (paper_1004_0023_gb300/estimators.py), checked
on oracle runs against exact results: exact diagonalisation for the quantum energy, the
transfer-matrix moments for E and M, and the counters for the rates."""
import numpy as np

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
