"""Create-time plan autotuning: candidate plans are timed on a continuous run, the context
is reset to its initial state, and the result is bit for bit the oracle's whichever plan
won; the choice is cached per shape."""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import instances
from paper_1004_0023_gb300 import pt

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _lib(libpt):
    return libpt


def _problem(n, P, R, seed):
    rng = np.random.default_rng(seed)
    return instances.make_problem("regular", rng, n=n, degree=3, P=P, R=R, n_sweeps=0,
                                  seed=instances.philox_seed(seed), ladder="geometric", g0=0.05, g1=4.0, T=0.02)


def _same(g, o):
    assert np.array_equal(g.read_state(), o.read_state())
    og, oo = g.obs(), o.obs()
    for k in oo:
        assert np.array_equal(np.asarray(og[k]), np.asarray(oo[k])), k


def test_autotuned_context_starts_from_the_initial_state_and_matches_the_oracle():
    # a shape no other test creates, so the first context really times its candidates
    prob = _problem(98, 64, 22, 4242)
    g = pt.PT.from_problem(prob)
    assert g.info.tuned_plans >= 2
    assert g.info.kernel_path in (2, 3, 5, 6, 7, 8, 9)
    o = Oracle.from_problem(prob, threads=THREADS)
    _same(g, o)  # the timed sweeps were undone
    g.run(150, 1)
    o.run(150, 1)
    _same(g, o)
    # the same shape again: the cached choice, nothing timed, the same plan
    h = pt.PT.from_problem(prob)
    assert h.info.tuned_plans == 0
    assert (h.info.kernel_path, h.info.threads_per_block) == (g.info.kernel_path, g.info.threads_per_block)
    h.run(150, 1)
    assert np.array_equal(h.read_state(), g.read_state())
    # autotuning off: the fixed automatic plan, same bits
    f = pt.PT.from_problem(prob, no_autotune=1)
    assert f.info.tuned_plans == 0 and f.info.kernel_path == 3
    f.run(150, 1)
    assert np.array_equal(f.read_state(), g.read_state())


def test_autotuned_short_ladder_may_take_the_one_cluster_plan():
    # R = 12 <= 16: path 9 (every chain's CTA in one cluster) is among the candidates
    prob = _problem(40, 32, 12, 4343)
    g = pt.PT.from_problem(prob)
    assert g.info.tuned_plans >= 2
    assert g.info.kernel_path in (2, 3, 7, 8, 9)
    o = Oracle.from_problem(prob, threads=THREADS)
    _same(g, o)
    g.run(200, 1)
    o.run(200, 1)
    _same(g, o)
