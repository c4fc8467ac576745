"""The paper-style multi-threaded CPU Parallel Tempering (cpu_pt/, Sec. 4, Figs. 4-5)
against the oracle: the same Markov chain, so bit-identical spins, E, M, statistics,
counters and rung permutation, for every thread count (its work pool hands chains out in a
data-dependent order, hardest first, which must never change a result)."""
import numpy as np
import pytest

from cpu_pt import CpuPT
from oracle import Oracle
from paper_1004_0023_gb300 import instances


def _same(a, b, where):
    assert np.array_equal(a.read_state(), b.read_state()), where
    oa, ob = a.obs(), b.obs()
    for k in ob:
        assert np.array_equal(np.asarray(oa[k]), np.asarray(ob[k])), (where, k)


CASES = {
    "line_p4_r3": instances.tiny_problem(3, [(0, 1), (1, 2)], [1, -2], [1, 0, -1], 4, [0.7, 1.0, 1.4],
                                         [0.9, 1.2, 1.6], seed=11),
    "pair_p2_r2": instances.tiny_problem(2, [(0, 1)], [2], [1, -1], 2, [0.5, 1.0], [0.5, 1.5], seed=12),
    "single_rung_p6": instances.tiny_problem(4, [(0, 1), (2, 3)], [1, -1], [1, -1, 0, 2], 6, [0.8], [1.1], seed=13),
    "classical_p1_r4": instances.tiny_problem(5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)], [1, -2, 1, -1, 2],
                                              [0, 1, 0, -1, 0], 1, [0.4, 0.8, 1.5, 3.0], [0, 0, 0, 0], seed=14),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("threads", [1, 2, 5])
def test_tiny_problems_equal_the_oracle(name, threads):
    prob = CASES[name]
    o = Oracle.from_problem(prob)
    c = CpuPT(prob, o.flip_table(), o.swap_coef(), threads=threads)
    _same(c, o, "initial")
    for s in range(12):
        c.run(1, 1)
        o.run(1, 1)
        _same(c, o, "sweep %d" % (s + 1))
    for n, sps in ((200, 3), (7, 0), (31, 4)):
        c.run(n, sps)
        o.run(n, sps)
        _same(c, o, "run(%d, %d)" % (n, sps))


@pytest.mark.parametrize("name,threads,sweeps", [("regular3_n16_p32_r16", 4, 300), ("regular3_n256_p64_r64", 8, 30),
                                                 ("classical_regular3_n256_r64", 3, 100)])
def test_workloads_equal_the_oracle(name, threads, sweeps):
    prob = instances.workload(name, 2)
    o = Oracle.from_problem(prob, threads=4)
    c = CpuPT.from_problem(prob, threads=threads)  # tables from the library's host helper
    c.run(sweeps, 1)
    o.run(sweeps, 1)
    _same(c, o, name)
    c.close()
    o.close()
