"""GPU path (through the C ABI) against the CPU oracle: bit-exact spins, integer E and M,
int64 statistics, counters and the rung permutation, at many checkpoints.

Tolerance is zero: integer couplings keep every quantity exact, the Metropolis table is
the same FP64-built uint32 table on both sides, random numbers are the same Philox4x32-10
counters, and the swap exp is the same sequence of IEEE operations.
"""
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import instances
from paper_1004_0023_gb300 import pt

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def assert_same(g, o, where=""):
    xs_g, xs_o = g.read_state(), o.read_state()
    if not np.array_equal(xs_g, xs_o):
        bad = np.argwhere(xs_g != xs_o)
        raise AssertionError("%s: %d spins differ, first (rung, site, copy) = %s" % (where, len(bad), bad[:5].tolist()))
    og, oo = g.obs(), o.obs()
    for k in oo:
        assert np.array_equal(np.asarray(og[k]), np.asarray(oo[k])), (where, k, og[k], oo[k])


def both(prob, threads=THREADS, **kw):
    okw = {k: v for k, v in kw.items() if k in ("flip_thr", "swap_coef")}
    # (the oracle takes no layout options)
    return pt.PT.from_problem(prob, **kw), Oracle.from_problem(prob, threads=threads, **okw)


@pytest.fixture(scope="module", autouse=True)
def _lib(libpt):
    return libpt


TINY = {
    "line_p4_r3": instances.tiny_problem(3, [(0, 1), (1, 2)], [1, -2], [1, 0, -1], 4, [0.7, 1.0, 1.4],
                                         [0.9, 1.2, 1.6], seed=11),
    "single_spin_p2_r2": instances.tiny_problem(1, [], [], [1], 2, [0.5, 1.0], [0.5, 1.5], seed=12),
    "no_edges_p6_r1": instances.tiny_problem(4, [], [], [1, -1, 0, 2], 6, [0.8], [1.1], seed=13),
    "prism_p10_r4": instances.tiny_problem(6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (0, 3), (1, 4), (2, 5)],
                                           [1, -2, 1, 2, -1, -1, 1, -2, 2], [1, 0, -1, 0, 1, 0], 10,
                                           [0.6, 0.8, 1.1, 1.5], [0.4, 0.8, 1.4, 2.2], seed=14),
    # packed path, 4 neighbour slots (degree 3 + h)
    "prism_p8_r3": instances.tiny_problem(6, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (0, 3), (1, 4), (2, 5)],
                                          [2, -1, 1, -2, 1, 1, -1, 2, -2], [0, 1, 0, -1, 1, 0], 8,
                                          [0.5, 0.9, 1.6], [0.6, 1.0, 1.8], seed=16),
    # packed path, 8 neighbour slots (degree 7 + h), P=16
    "complete8_p16_r4": instances.tiny_problem(
        8, [(i, j) for i in range(8) for j in range(i + 1, 8)],
        [((i * 5 + j * 3) % 5) - 2 or 2 for i in range(8) for j in range(i + 1, 8)],
        [1, 0, -1, 2, 0, -2, 1, 0], 16, [0.4, 0.7, 1.2, 2.0], [0.3, 0.7, 1.3, 2.4], seed=17),
    # byte-wise path (degree 9)
    "complete10_p12_r5": instances.tiny_problem(
        10, [(i, j) for i in range(10) for j in range(i + 1, 10)],
        [((i * 7 + j * 3) % 5) - 2 or 1 for i in range(10) for j in range(i + 1, 10)],
        [0, 1, -1, 2, 0, 0, 1, -2, 0, 1], 12, [0.5, 0.7, 1.0, 1.4, 2.0], [0.3, 0.6, 1.0, 1.5, 2.5], seed=15),
}


@pytest.mark.parametrize("name", sorted(TINY))
def test_tiny_problems_every_sweep(name):
    prob = TINY[name]
    g, o = both(prob)
    assert_same(g, o, "initial")
    for s in range(1, 41):
        g.run(1, 1)
        o.run(1, 1)
        assert_same(g, o, "sweep %d" % s)
    g.run(500, 3)
    o.run(500, 3)
    assert_same(g, o, "after 500 more")


def test_small_workload_full_length():
    """Random 3-regular N=16, P=32, R=16, linear Gamma 0.1..3.0 at T=0.05, 10^4 sweeps,
    one swap pass per sweep; checked every 500 sweeps."""
    prob = instances.workload("regular3_n16_p32_r16", 1)
    g, o = both(prob)
    for chunk in range(prob.n_sweeps // 500):
        g.run(500, 1)
        o.run(500, 1)
        assert_same(g, o, "sweep %d" % (500 * (chunk + 1)))


def test_medium_workload_full_length():
    """Random 3-regular N=256, P=64, R=64, geometric Gamma 0.05..4.0 at T=0.02, 2000 sweeps;
    bit-exact state check every 100 sweeps."""
    prob = instances.workload("regular3_n256_p64_r64", 1)
    g, o = both(prob)
    for chunk in range(prob.n_sweeps // 100):
        g.run(100, 1)
        o.run(100, 1)
        assert_same(g, o, "sweep %d" % (100 * (chunk + 1)))


@pytest.mark.parametrize("producers", [0, 32])
def test_small_workload_on_path_9(producers):
    """N=16, P=32, R=16 with all 16 chains' CTAs in one cluster and the swap mailboxes in
    shared memory (random words inline, or from a producer warp): full length, checked every
    1000 sweeps."""
    prob = instances.workload("regular3_n16_p32_r16", 1)
    g, o = both(prob, kernel_path=9, producer_threads=producers)
    assert g.info.kernel_path == 9
    for chunk in range(prob.n_sweeps // 1000):
        g.run(1000, 1)
        o.run(1000, 1)
        assert_same(g, o, "sweep %d" % (1000 * (chunk + 1)))


@pytest.mark.parametrize("R,cluster", [(1, 0), (5, 2), (17, 0), (20, 8)])
def test_classical_ladders_of_any_length_on_path_10(R, cluster):
    """Path 10 with one chain, with a last CTA holding fewer chains than the others (5 = 4 + 1,
    17 = 16 + 1, 20 = 3 x 8 - 4 idle slots), and the default cluster."""
    ladder_T = np.geomspace(0.4, 3.0, R)
    edges = [(i, (i + 1) % 24) for i in range(24)] + [(i, (i + 12) % 24) for i in range(12)]
    J = [((3 * i + 1) % 5) - 2 or 1 for i in range(len(edges))]
    h = [((5 * i) % 3) - 1 for i in range(24)]
    prob = instances.tiny_problem(24, edges, J, h, 1, ladder_T, np.zeros(R), seed=600 + R)
    g, o = both(prob, kernel_path=10, cluster_size=cluster)
    assert g.info.kernel_path == 10
    for s in range(12):
        g.run(1, 1)
        o.run(1, 1)
        assert_same(g, o, "sweep %d" % (s + 1))
    g.run(300, 2)
    o.run(300, 2)
    assert_same(g, o, "after 300 more")


def test_classical_partner_that_never_publishes_times_out_on_path_10():
    """Path 10: the chain on rung 3 withholds its publication; its partner's bounded wait in
    shared memory runs out, every CTA of the cluster reaches the closing cluster barrier, and
    the call reports PT_ETIMEDOUT; the device stays usable."""
    prob = instances.workload("classical_regular3_n256_r64", 2)
    g = pt.PT.from_problem(prob, wait_timeout_ms=200, test_withhold_rung=3, kernel_path=10)
    g.run(4, 1)
    with pytest.raises(pt.PTError) as e:
        g.sync()
    assert e.value.code == pt.PT_ETIMEDOUT
    g.close()
    h, o = both(prob, kernel_path=10)
    h.run(50, 1)
    o.run(50, 1)
    assert_same(h, o, "after timeout")


def test_path_10_needs_classical_chains():
    prob = instances.workload("regular3_n16_p32_r16", 1)  # P = 32
    with pytest.raises(pt.PTError) as e:
        pt.PT.from_problem(prob, kernel_path=10)
    assert e.value.code == pt.PT_EINVAL
    classical = instances.workload("classical_regular3_n256_r64", 1)  # R = 64
    # (cluster_size 1 puts all 64 chains on one CTA, which needs a multiple of 64 threads)
    for kw in (dict(cluster_size=17), dict(threads_per_block=48), dict(threads_per_block=1024),
               dict(cluster_size=1, threads_per_block=32)):
        with pytest.raises(pt.PTError) as e:
            pt.PT.from_problem(classical, kernel_path=10, **kw)
        assert e.value.code == pt.PT_EINVAL, kw


def test_path_9_needs_the_ladder_in_one_cluster():
    prob = instances.workload("regular3_n256_p64_r64", 1)  # R = 64 > 16
    with pytest.raises(pt.PTError) as e:
        pt.PT.from_problem(prob, kernel_path=9)
    assert e.value.code == pt.PT_EINVAL
    small = instances.workload("regular3_n16_p32_r16", 1)
    for kw in (dict(threads_per_block=32), dict(threads_per_block=512), dict(producer_threads=16),
               dict(producer_threads=128)):
        with pytest.raises(pt.PTError) as e:
            pt.PT.from_problem(small, kernel_path=9, **kw)
        assert e.value.code == pt.PT_EINVAL, kw


def test_medium_workload_on_path_8():
    """N=256, P=64, R=64 with each chain's random words made by a second CTA of its cluster
    (path 8), 384 and 512 threads, checked every 200 sweeps."""
    prob = instances.workload("regular3_n256_p64_r64", 1)
    for th in (384, 512):
        g, o = both(prob, kernel_path=8, threads_per_block=th)
        assert g.info.kernel_path == 8
        for chunk in range(3):
            g.run(200, 1)
            o.run(200, 1)
            assert_same(g, o, "threads %d sweep %d" % (th, 200 * (chunk + 1)))
        g.close()
        o.close()


@pytest.mark.parametrize("seed_index", [2, 3])
def test_medium_workload_other_seeds(seed_index):
    prob = instances.workload("regular3_n256_p64_r64", seed_index)
    g, o = both(prob)
    g.run(200, 1)
    o.run(200, 1)
    assert_same(g, o, "seed %d" % seed_index)


def test_layouts_and_swap_modes_give_identical_bits():
    prob = instances.workload("regular3_n16_p32_r16", 2)
    ref = None
    for kw in (dict(threads_per_block=32), dict(threads_per_block=128), dict(threads_per_block=512),
               dict(swap_mode=2), dict(swap_mode=1, threads_per_block=64),
               dict(kernel_path=1), dict(kernel_path=1, threads_per_block=96), dict(kernel_path=2),
               dict(kernel_path=2, threads_per_block=64), dict(kernel_path=3), dict(kernel_path=3, producer_threads=32),
               dict(kernel_path=3, threads_per_block=256, producer_threads=160), dict(kernel_path=3, swap_mode=2),
               dict(kernel_path=4), dict(kernel_path=4, threads_per_block=32), dict(kernel_path=4, swap_mode=2),
               dict(kernel_path=3, threads_per_block=64, producer_threads=32),
               dict(test_exact_swaps=1), dict(test_exact_swaps=1, swap_mode=2),
               dict(kernel_path=8), dict(kernel_path=8, threads_per_block=384), dict(kernel_path=8, swap_mode=2),
               dict(kernel_path=9), dict(kernel_path=9, threads_per_block=64),
               dict(kernel_path=9, threads_per_block=256, producer_threads=64),
               dict(kernel_path=9, producer_threads=32), dict(kernel_path=9, swap_mode=2)):
        g = pt.PT.from_problem(prob, **kw)
        g.run(300, 1)
        g.run(77, 5)
        cur = (g.read_state(), g.obs())
        if ref is None:
            ref = cur
        else:
            assert np.array_equal(cur[0], ref[0]), kw
            for k in ref[1]:
                assert np.array_equal(np.asarray(cur[1][k]), np.asarray(ref[1][k])), (kw, k)


@pytest.mark.parametrize("path", [1, 2, 3, 4, 8])
def test_medium_workload_each_kernel_path(path):
    prob = instances.workload("regular3_n256_p64_r64", 4)
    g, o = both(prob, kernel_path=path)
    assert g.info.kernel_path == path
    g.run(150, 1)
    o.run(150, 1)
    assert_same(g, o, "path %d" % path)


@pytest.mark.parametrize("path", [1, 2, 3, 4, 8, 9])
@pytest.mark.parametrize("name", ["prism_p8_r3", "complete8_p16_r4"])
def test_tiny_packed_problems_each_path(name, path):
    prob = TINY[name]
    g, o = both(prob, kernel_path=path)
    for s in range(30):
        g.run(1, 1)
        o.run(1, 1)
        assert_same(g, o, "sweep %d" % (s + 1))
    g.run(300, 2)
    o.run(300, 2)
    assert_same(g, o, "after 300 more")


def test_lattice_workload_bit_packed():
    """K4,4 cells on a 16x16 grid (N=2048), P=128, R=96: one int8 chain (256 KiB) does not
    fit in shared memory, so the automatic plan holds it at one bit per copy; checked every
    50 sweeps over the first 200 and at the end of the 500-sweep run."""
    prob = instances.workload("chimera16_n2048_p128_r96", 1)
    g, o = both(prob)
    assert g.info.kernel_path == 4
    for chunk in range(4):
        g.run(50, 1)
        o.run(50, 1)
        assert_same(g, o, "sweep %d" % (50 * (chunk + 1)))
    g.run(prob.n_sweeps - 200, 1)
    o.run(prob.n_sweeps - 200, 1)
    assert_same(g, o, "sweep %d" % prob.n_sweeps)


@pytest.mark.parametrize("path", [2, 3, 4, 8, 9])
@pytest.mark.parametrize("P", [8, 24, 136])
def test_packed_row_lengths(P, path):
    """Rows of 8, 24 and 136 copies (1, 3 and 17 bytes bit-packed): the periodic Trotter
    neighbour across the row's ends, ragged 16-byte padding of the chain, and row sizes that
    are not powers of two; degree-6 lattice with fields and degree-3 graph."""
    rng = np.random.default_rng(P)
    for graph, kw in (("chimera", dict(rows=2, cols=3)), ("regular", dict(n=38, degree=3))):
        prob = instances.make_problem(graph, rng, P=P, R=5, n_sweeps=0, seed=instances.philox_seed(500 + P),
                                      ladder="geometric", g0=0.1, g1=3.0, T=0.2, J=(-3, -1, 2, 4), h=(-2, 0, 1), **kw)
        g, o = both(prob, kernel_path=path)
        for s in range(6):
            g.run(1, 1)
            o.run(1, 1)
            assert_same(g, o, "%s P=%d sweep %d" % (graph, P, s + 1))
        g.run(200, 3)
        o.run(200, 3)
        assert_same(g, o, "%s P=%d after 200 more" % (graph, P))


@pytest.mark.parametrize("kw", [dict(kernel_path=1), dict(kernel_path=10, cluster_size=1),
                                dict(kernel_path=10, cluster_size=2), dict(kernel_path=10, cluster_size=3),
                                dict(kernel_path=10, cluster_size=1, threads_per_block=32), dict()])
def test_classical_tiny_problem_every_sweep(kw):
    """Classical parallel tempering (P = 1, Gamma = 0, temperature ladder) on the byte-wise
    kernel and on path 10 (three chains on one CTA with a fourth, idle slot; on two CTAs of two
    and one; on three CTAs): bits after every sweep, then after 500 more with a swap every
    third sweep."""
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (0, 3), (1, 4)]
    prob = instances.tiny_problem(6, edges, [1, -2, 1, -1, 2, -1, 1, -2], [1, 0, -1, 0, 1, 0], 1,
                                  [0.7, 1.4, 3.0], [0.0, 0.0, 0.0], seed=31)
    g, o = both(prob, **kw)
    assert g.info.kernel_path == kw.get("kernel_path", g.info.kernel_path)
    assert g.info.kernel_path in (1, 10)
    for s in range(30):
        g.run(1, 1)
        o.run(1, 1)
        assert_same(g, o, "sweep %d" % (s + 1))
    g.run(500, 3)
    o.run(500, 3)
    assert_same(g, o, "after 500 more")


@pytest.mark.parametrize("kw", [dict(), dict(kernel_path=1), dict(kernel_path=10),
                                dict(kernel_path=10, cluster_size=16)])
def test_classical_workload_full_length(kw):
    """Random 3-regular N=256, P=1, R=64 temperatures geometric 0.1..3.0, 2000 sweeps with a
    swap pass after every sweep; checked every 200 sweeps: the autotuned plan, the byte-wise
    kernel, and path 10 with 16 chains on each of 4 CTAs and 4 chains on each of 16."""
    prob = instances.workload("classical_regular3_n256_r64", 1)
    g, o = both(prob, **kw)
    for chunk in range(prob.n_sweeps // 200):
        g.run(200, 1)
        o.run(200, 1)
        assert_same(g, o, "sweep %d" % (200 * (chunk + 1)))
    assert np.all(np.asarray(g.obs()["M"]) == prob.n)


def test_exact_swap_rule_and_fast_pre_decision_agree_on_the_medium_workload():
    """Every swap decided by the FP32 pre-decision equals the FP64 rule (both vs the oracle)."""
    prob = instances.workload("regular3_n256_p64_r64", 5)
    a = pt.PT.from_problem(prob)
    b = pt.PT.from_problem(prob, test_exact_swaps=1)
    o = Oracle.from_problem(prob, threads=THREADS)
    for x in (a, b):
        x.run(400, 1)
    o.run(400, 1)
    assert_same(a, o, "pre-decided swaps")
    assert_same(b, o, "exact swaps")


def test_run_equals_sweep_and_swap_calls():
    prob = instances.workload("regular3_n16_p32_r16", 3)
    a = pt.PT.from_problem(prob)
    b = pt.PT.from_problem(prob)
    a.run(60, 3)
    for _ in range(20):
        b.sweep(3)
        b.swap()
    assert np.array_equal(a.read_state(), b.read_state())
    oa, ob = a.obs(), b.obs()
    for k in oa:
        assert np.array_equal(np.asarray(oa[k]), np.asarray(ob[k])), k


def test_checkpoint_restore_continues_bit_for_bit():
    """A checkpoint of one context restored into a fresh context of the same problem (after
    swaps have moved the chains between rungs) continues exactly like the original; also
    after restoring an older checkpoint into a context that ran further."""
    prob = instances.workload("regular3_n16_p32_r16", 5)
    a = pt.PT.from_problem(prob)
    a.run(300, 1)
    state, ob = a.checkpoint()
    assert not np.array_equal(ob["replica_at"], np.arange(prob.R))  # some swaps were accepted
    b = pt.PT.from_problem(prob)
    b.run(1000, 1)  # further than the checkpoint: its mailboxes hold later passes
    b.restore(state, ob)
    assert_same(b, _Frozen(state, ob), "right after restore")
    a.run(250, 1)
    b.run(250, 1)
    assert_same(b, _Frozen(*a.checkpoint()), "250 sweeps after restore")
    o = Oracle.from_problem(prob, threads=THREADS)
    o.run(550, 1)
    assert_same(b, o, "vs oracle")
    with pytest.raises(pt.PTError) as e:
        bad = dict(ob)
        bad["replica_at"] = np.zeros(prob.R, np.int32)
        b.restore(state, bad)
    assert e.value.code == pt.PT_EINVAL


class _Frozen:
    """A checkpoint seen through the read_state / obs interface of assert_same."""

    def __init__(self, state, ob):
        self._s, self._o = state, ob

    def read_state(self):
        return self._s

    def obs(self):
        return self._o


def test_tables_read_back_equal_oracle():
    prob = instances.workload("regular3_n256_p64_r64", 1)
    g, o = both(prob)
    thr, coef = g.tables()
    assert np.array_equal(thr, o.flip_table())
    assert np.array_equal(coef.view(np.uint64), o.swap_coef().view(np.uint64))


def test_all_accept_table_and_write_state():
    prob = instances.workload("regular3_n16_p32_r16", 4)
    lmax = Oracle.from_problem(prob).lmax
    thr = np.full((prob.R, 2 * lmax + 1, 3), 0xFFFFFFFF, np.uint32)
    g, o = both(prob, flip_thr=thr)
    rng = np.random.default_rng(0)
    x = np.where(rng.random((prob.R, prob.n, prob.P)) < 0.5, -1, 1).astype(np.int8)
    g.write_state(x)
    o.write_state(x)
    assert_same(g, o, "written")
    g.sweep(1)
    o.sweep(1)
    assert np.array_equal(g.read_state(), -x)
    assert_same(g, o, "negated")


def test_invalid_arguments_are_rejected():
    prob = instances.workload("regular3_n16_p32_r16", 1)
    with pytest.raises(pt.PTError) as e:
        pt.PT(prob.n, prob.ei, prob.ej, prob.J, prob.h, 3, prob.T, prob.gamma, 1)
    assert e.value.code == pt.PT_EINVAL
    bad_J = prob.J.copy()
    bad_J[0] = 0
    with pytest.raises(pt.PTError):
        pt.PT(prob.n, prob.ei, prob.ej, bad_J, prob.h, prob.P, prob.T, prob.gamma, 1)
    g = pt.PT.from_problem(prob)
    with pytest.raises(pt.PTError) as e:
        g.write_state(np.zeros((prob.R, prob.n, prob.P), np.int8))
    assert e.value.code == pt.PT_EINVAL
    with pytest.raises(pt.PTError) as e:
        g.sweep(1 << 40)
    assert e.value.code == pt.PT_EOVERFLOW
    g.run(10, 1)  # still usable after argument errors


@pytest.mark.parametrize("path", [0, 1, 2, 3, 4, 8, 9])
def test_partner_that_never_publishes_times_out_without_fault(path):
    """The chain on rung 3 withholds its mailbox: its partner's bounded wait runs out, the
    call reports PT_ETIMEDOUT, and the device stays usable for a new context. On every
    one-CTA kernel, with sweeps left after the one whose wait gave up: the CTA that gave up
    leaves at the next barrier without touching its random-word buffers; on path 8 its
    random-word CTA learns at that same cluster barrier and leaves with it; on path 9 every
    CTA of the cluster reaches the closing cluster barrier (each wait is bounded)."""
    prob = instances.workload("regular3_n16_p32_r16", 5)
    g = pt.PT.from_problem(prob, wait_timeout_ms=200, test_withhold_rung=3, swap_mode=1, kernel_path=path)
    g.run(4, 1)
    with pytest.raises(pt.PTError) as e:
        g.sync()
    assert e.value.code == pt.PT_ETIMEDOUT
    with pytest.raises(pt.PTError):  # sticky
        g.run(1, 1)
    g.close()
    h, o = both(prob)
    h.run(50, 1)
    o.run(50, 1)
    assert_same(h, o, "after timeout")


def test_largest_trotter_stack_and_largest_resident_chain():
    """P = 4096, the largest P accepted: 512 words per parity, more word columns than a CTA
    has threads, so the level loop runs in its flat unit order. And N = 4096 sites at P = 16
    (64 KiB of int8 chain per replica). Both bit-exact with the oracle."""
    rng = np.random.default_rng(4096)
    big_p = instances.make_problem("regular", rng, n=6, degree=3, P=4096, R=3, n_sweeps=0,
                                   seed=instances.philox_seed(4096), ladder="geometric", g0=0.1, g1=3.0, T=0.2)
    g, o = both(big_p)
    for s in range(3):
        g.run(1, 1)
        o.run(1, 1)
        assert_same(g, o, "P=4096 sweep %d" % (s + 1))
    g.run(40, 2)
    o.run(40, 2)
    assert_same(g, o, "P=4096 after 40 more")
    big_n = instances.make_problem("regular", rng, n=4096, degree=3, P=16, R=4, n_sweeps=0,
                                   seed=instances.philox_seed(4097), ladder="geometric", g0=0.1, g1=3.0, T=0.2)
    g, o = both(big_n)
    g.run(30, 1)
    o.run(30, 1)
    assert_same(g, o, "N=4096")


def test_chain_too_large_for_any_layout_is_rejected():
    """A chain no layout can hold in one SM's shared memory is refused at create with
    PT_EINVAL (nothing is launched), and the device stays usable."""
    rng = np.random.default_rng(5)
    huge = instances.make_problem("regular", rng, n=60000, degree=3, P=64, R=2, n_sweeps=0,
                                  seed=instances.philox_seed(5), ladder="geometric", g0=0.1, g1=3.0, T=0.2)
    with pytest.raises(pt.PTError) as e:
        pt.PT.from_problem(huge)
    assert e.value.code == pt.PT_EINVAL
    prob = instances.workload("regular3_n16_p32_r16", 1)
    g, o = both(prob)
    g.run(20, 1)
    o.run(20, 1)
    assert_same(g, o, "after a refused create")


def test_more_chains_than_fit_at_once():
    """R = 200 chains of the N=256, P=64 workload. With the producer-warp kernel one chain
    fills an SM, so not every chain can be resident, and swap passes run as separate launches
    between sweep launches. The automatic plan times only candidates whose chains all fit
    (the inline-word kernel: several CTAs per SM) and so swaps inside one launch. Both give
    the oracle's bits."""
    spec = dict(instances.WORKLOADS["regular3_n256_p64_r64"])
    spec["R"] = 200
    rng = np.random.default_rng(200)
    prob = instances.make_problem(spec.pop("graph"), rng, seed=instances.philox_seed(200), name="r200", **spec)
    o = Oracle.from_problem(prob, threads=THREADS)
    o.run(20, 1)
    for kw in (dict(kernel_path=3), dict()):
        g = pt.PT.from_problem(prob, **kw)
        assert bool(g.info.cooperative) == (not kw)
        g.run(20, 1)
        assert_same(g, o, "R=200 %s" % kw)
        g.close()
