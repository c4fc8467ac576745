"""Path 7 (every chain of one problem resident on one thread-block cluster, swap passes
decided in shared memory) against the CPU oracle: bit-exact spins, E, M, statistics,
counters and the rung permutation, for every cluster size and chain-group width that holds
the chains, through pt_run, pt_sweep + pt_swap, and with sweep counts that are not a
multiple of the swap interval. The tolerance is zero, as for every other plan."""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import instances, pt

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _lib(libpt):
    return libpt


def _same(g, o, where):
    xs_g, xs_o = g.read_state(), o.read_state()
    if not np.array_equal(xs_g, xs_o):
        bad = np.argwhere(xs_g != xs_o)
        raise AssertionError("%s: %d spins differ, first %s" % (where, len(bad), bad[:5].tolist()))
    og, oo = g.obs(), o.obs()
    for k in oo:
        assert np.array_equal(np.asarray(og[k]), np.asarray(oo[k])), (where, k)


def test_small_workload_full_length_on_one_cluster():
    """N=16, P=32, R=16 (all 16 chains, 8 KiB, in one CTA), 10^4 sweeps, checked every 1000."""
    prob = instances.workload("regular3_n16_p32_r16", 1)
    g = pt.PT.from_problem(prob, kernel_path=7)
    o = Oracle.from_problem(prob, threads=THREADS)
    assert g.info.kernel_path == 7
    for chunk in range(prob.n_sweeps // 1000):
        g.run(1000, 1)
        o.run(1000, 1)
        _same(g, o, "sweep %d" % (1000 * (chunk + 1)))


@pytest.mark.parametrize("cluster,group", [(1, 32), (1, 64), (1, 0), (2, 32), (2, 128), (4, 0), (8, 32), (16, 32)])
def test_cluster_sizes_and_group_widths(cluster, group):
    prob = instances.workload("regular3_n16_p32_r16", 3)
    g = pt.PT.from_problem(prob, kernel_path=7, cluster_size=cluster, group_threads=group)
    o = Oracle.from_problem(prob, threads=THREADS)
    for s in range(5):
        g.run(1, 1)
        o.run(1, 1)
        _same(g, o, "K=%d g=%d sweep %d" % (cluster, group, s + 1))
    g.run(400, 1)
    o.run(400, 1)
    _same(g, o, "K=%d g=%d after 400 more" % (cluster, group))
    g.run(101, 4)  # 25 passes and a tail sweep
    o.run(101, 4)
    _same(g, o, "K=%d g=%d tail" % (cluster, group))


@pytest.mark.parametrize("cluster", [8, 16])
def test_medium_workload_on_a_cluster(cluster):
    """N=256, P=64, R=64: 64 chains of 16 KiB over 8 or 16 CTAs of one cluster (4 CTAs would need 256 KiB each)."""
    prob = instances.workload("regular3_n256_p64_r64", 5)
    g = pt.PT.from_problem(prob, kernel_path=7, cluster_size=cluster)
    o = Oracle.from_problem(prob, threads=THREADS)
    for chunk in range(3):
        g.run(50, 1)
        o.run(50, 1)
        _same(g, o, "K=%d sweep %d" % (cluster, 50 * (chunk + 1)))


def test_sweep_and_swap_calls_and_tiny_problems():
    # pt_sweep / pt_swap interleaved with pt_run on path 7
    prob = instances.workload("regular3_n16_p32_r16", 4)
    g = pt.PT.from_problem(prob, kernel_path=7, cluster_size=2)
    o = Oracle.from_problem(prob, threads=THREADS)
    for _ in range(7):
        g.sweep(3)
        o.sweep(3)
        g.swap()
        o.swap()
    g.run(33, 2)
    o.run(33, 2)
    g.sweep(5)
    o.sweep(5)
    _same(g, o, "mixed calls")
    # degree-7 problem (8 neighbour slots), P = 16, R = 4, and R = 1 (no pairs)
    p8 = instances.tiny_problem(8, [(i, j) for i in range(8) for j in range(i + 1, 8)],
                                [((i * 5 + j * 3) % 5) - 2 or 2 for i in range(8) for j in range(i + 1, 8)],
                                [1, 0, -1, 2, 0, -2, 1, 0], 16, [0.4, 0.7, 1.2, 2.0], [0.3, 0.7, 1.3, 2.4], seed=17)
    p1 = instances.tiny_problem(3, [(0, 1), (1, 2)], [1, -2], [1, 0, -1], 8, [0.7], [0.9], seed=18)
    for prob in (p8, p1):
        g = pt.PT.from_problem(prob, kernel_path=7)
        o = Oracle.from_problem(prob)
        for s in range(20):
            g.run(1, 1)
            o.run(1, 1)
            _same(g, o, "%s sweep %d" % (prob.name, s + 1))
        g.run(300, 3)
        o.run(300, 3)
        _same(g, o, "%s after 300 more" % prob.name)


def test_checkpoint_restore_onto_path_7():
    prob = instances.workload("regular3_n16_p32_r16", 6)
    a = pt.PT.from_problem(prob, kernel_path=2)
    a.run(250, 1)
    state, obs = a.checkpoint()
    b = pt.PT.from_problem(prob, kernel_path=7)
    b.restore(state, obs)
    a.run(300, 1)
    b.run(300, 1)
    assert np.array_equal(a.read_state(), b.read_state())
    oa, ob = a.obs(), b.obs()
    for k in oa:
        assert np.array_equal(np.asarray(oa[k]), np.asarray(ob[k])), k


def test_path_7_argument_checks():
    prob = instances.workload("regular3_n16_p32_r16", 1)
    for kw in (dict(kernel_path=7, group_threads=48), dict(kernel_path=7, group_threads=1024),
               dict(kernel_path=7, cluster_size=17), dict(kernel_path=7, threads_per_block=256),
               dict(kernel_path=7, test_withhold_rung=2)):
        with pytest.raises(pt.PTError) as e:
            pt.PT.from_problem(prob, **kw)
        assert e.value.code == pt.PT_EINVAL, kw
    big = instances.workload("chimera16_n2048_p128_r96", 1)  # int8 chains of 256 KiB fit no CTA
    with pytest.raises(pt.PTError) as e:
        pt.PT.from_problem(big, kernel_path=7)
    assert e.value.code == pt.PT_EINVAL
