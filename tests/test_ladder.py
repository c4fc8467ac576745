"""Ladder adaptation (paper_1004_0023_gb300/ladder.py): fixed point, direction of the moves,
and on oracle runs the worst pair's acceptance rises."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import estimators, instances, ladder


def test_equal_acceptance_is_a_fixed_point_and_ends_stay():
    x = np.geomspace(0.05, 4.0, 9)
    assert np.allclose(ladder.adapt(x, np.full(8, 0.3)), x)
    y = ladder.adapt(x, np.linspace(0.05, 0.9, 8))
    assert y[0] == x[0] and y[-1] == x[-1] and np.all(np.diff(y) > 0)


def test_rungs_move_towards_a_bottleneck():
    x = np.linspace(1.0, 2.0, 6)
    acc = np.array([0.8, 0.8, 0.02, 0.8, 0.8])  # the middle pair hardly ever swaps
    y = ladder.adapt(x, acc)
    # the middle gap shrinks, the others grow
    assert (y[3] - y[2]) < (x[3] - x[2])
    assert (y[1] - y[0]) > (x[1] - x[0]) and (y[5] - y[4]) > (x[5] - x[4])


def test_bad_inputs_are_rejected():
    with pytest.raises(ValueError):
        ladder.adapt([1.0, 2.0, 3.0], [0.5])
    with pytest.raises(ValueError):
        ladder.adapt([1.0, 3.0, 2.0], [0.5, 0.5])


def test_adaptation_raises_the_worst_swap_rate_on_oracle_runs():
    """Classical ladder with its rungs crowded at high T: after two rounds of adaptation the
    least accepting pair accepts more often (deterministic: fixed seeds)."""
    base = instances.make_problem("regular", np.random.default_rng(3), n=24, degree=3, P=1, R=8,
                                  ladder="temperature", g0=0.3, g1=3.0, n_sweeps=0, seed=instances.philox_seed(40))
    T = np.concatenate([[0.3], np.geomspace(1.5, 3.0, 7)])  # a large gap at the cold end
    prob = type(base)(**{**base.__dict__, "T": T})

    def rates(p):
        o = Oracle.from_problem(p)
        o.run(500, 1)
        start = o.obs()
        o.run(3000, 1)
        ob = o.obs()
        return estimators.swap_rate(ob, since=start), ob, start

    r0, ob, start = rates(prob)
    p1 = ladder.adapt_problem(prob, ob, since=start)
    r1, ob, start = rates(p1)
    p2 = ladder.adapt_problem(p1, ob, since=start)
    r2, _, _ = rates(p2)
    assert p2.T[0] == prob.T[0] and p2.T[-1] == prob.T[-1]
    assert max(r1.min(), r2.min()) > 2 * r0.min() + 0.01, (r0, r1, r2)
    assert np.ptp(r2) < 0.5 * np.ptp(r0), (r0, r2)  # acceptance evens out along the ladder
