"""The split sweep kernel (kernel_path 5: one chain on a cluster of two CTAs, each holding
half of the Trotter copies and recomputing the neighbouring half's first even word) against
the CPU oracle, bit for bit: spins, E, M, statistics, counters and the rung permutation.
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


def both(prob, **kw):
    return pt.PT.from_problem(prob, **kw), Oracle.from_problem(prob, threads=THREADS)


@pytest.fixture(scope="module", autouse=True)
def _lib(libpt):
    return libpt


@pytest.mark.parametrize("path", [5, 6])
def test_medium_workload_full_length_split(path):
    """Random 3-regular N=256, P=64, R=64, 2000 sweeps with a swap pass after each; state
    checked every 100 sweeps (random words produced ahead, path 5, or inline, path 6)."""
    prob = instances.workload("regular3_n256_p64_r64", 1)
    g, o = both(prob, kernel_path=path)
    assert g.info.kernel_path == path
    for chunk in range(prob.n_sweeps // 100):
        g.run(100, 1)
        o.run(100, 1)
        assert_same(g, o, "sweep %d" % (100 * (chunk + 1)))


@pytest.mark.parametrize("path", [5, 6])
@pytest.mark.parametrize("P", [16, 32, 48, 128])
def test_split_row_lengths(P, path):
    """W = P/16 = 1, 2, 3 and 8 words per parity and CTA (word columns 2..9), on a degree-6
    lattice with fields (eight neighbour slots) and a degree-3 graph (four); every sweep for
    six sweeps, then 200 more with a swap pass every third sweep."""
    rng = np.random.default_rng(1000 + P)
    for graph, kw in (("chimera", dict(rows=2, cols=3)), ("regular", dict(n=38, degree=3))):
        prob = instances.make_problem(graph, rng, P=P, R=5, n_sweeps=0, seed=instances.philox_seed(700 + P),
                                      ladder="geometric", g0=0.1, g1=3.0, T=0.2, J=(-3, -1, 2, 4), h=(-2, 0, 1), **kw)
        g, o = both(prob, kernel_path=path)
        for s in range(6):
            g.run(1, 1)
            o.run(1, 1)
            assert_same(g, o, "%s P=%d sweep %d" % (graph, P, s + 1))
        g.run(200, 3)
        o.run(200, 3)
        assert_same(g, o, "%s P=%d after 200 more" % (graph, P))


def test_split_layouts_sweeps_and_swap_modes_give_identical_bits():
    """Thread and producer counts, sweeps without swaps (no cooperative launch) and one
    launch per swap interval all give the bits of the one-CTA-per-chain kernel."""
    prob = instances.workload("regular3_n16_p32_r16", 2)
    ref = None
    for kw in (dict(kernel_path=3), dict(kernel_path=5), dict(kernel_path=5, producer_threads=32),
               dict(kernel_path=5, threads_per_block=256, producer_threads=64),
               dict(kernel_path=5, threads_per_block=512, producer_threads=256),
               dict(kernel_path=5, swap_mode=2), dict(kernel_path=6), dict(kernel_path=6, threads_per_block=384),
               dict(kernel_path=6, threads_per_block=64), dict(kernel_path=6, swap_mode=2)):
        g = pt.PT.from_problem(prob, **kw)
        g.run(300, 1)
        g.sweep(13)
        g.run(77, 5)
        cur = (g.read_state(), g.obs())
        if ref is None:
            ref = cur
        else:
            assert np.array_equal(cur[0], ref[0]), kw
            for k in ref[1]:
                assert np.array_equal(np.asarray(cur[1][k]), np.asarray(ref[1][k])), (kw, k)


def test_split_rejects_unsupported_shapes():
    prob = instances.workload("regular3_n16_p32_r16", 1)
    rng = np.random.default_rng(3)
    p24 = instances.make_problem("regular", rng, n=16, degree=3, P=24, R=4, seed=5)
    for path in (5, 6):
        with pytest.raises(pt.PTError) as e:
            pt.PT.from_problem(p24, kernel_path=path)
        assert e.value.code == pt.PT_EINVAL
    # P = 512: 33 word columns, more than the 32 consumer threads asked for
    p512 = instances.make_problem("regular", rng, n=4, degree=3, P=512, R=2, seed=6)
    with pytest.raises(pt.PTError) as e:
        pt.PT.from_problem(p512, kernel_path=5, threads_per_block=64, producer_threads=32)
    assert e.value.code == pt.PT_EINVAL
    pt.PT.from_problem(prob, kernel_path=5).close()


@pytest.mark.parametrize("path", [5, 6])
def test_split_partner_that_never_publishes_times_out_without_fault(path):
    """A withheld mailbox makes the bounded swap wait of both CTAs of the partner chain run
    out: the call reports PT_ETIMEDOUT, every CTA leaves through the same cluster barriers,
    and the device stays usable."""
    prob = instances.workload("regular3_n16_p32_r16", 5)
    g = pt.PT.from_problem(prob, wait_timeout_ms=200, test_withhold_rung=3, swap_mode=1, kernel_path=path)
    g.run(4, 1)
    with pytest.raises(pt.PTError) as e:
        g.sync()
    assert e.value.code == pt.PT_ETIMEDOUT
    g.close()
    h, o = both(prob, kernel_path=path)
    h.run(50, 1)
    o.run(50, 1)
    assert_same(h, o, "after timeout")


def test_auto_plan_splits_chains_that_do_not_fit_one_cta():
    """N=256, P=128, R=64: one CTA cannot hold a chain with a sweep of produced random words,
    two can, and 64 clusters fit the GPU, so the split kernels are among the automatic plan's
    timed candidates (with the one-CTA inline-word kernels); whichever wins, the bits equal
    the oracle's and the inline-word kernel's."""
    spec = dict(instances.WORKLOADS["regular3_n256_p64_r64"])
    spec["P"] = 128
    rng = np.random.default_rng(9)
    prob = instances.make_problem(spec.pop("graph"), rng, seed=instances.philox_seed(9), name="p128", **spec)
    g, o = both(prob)
    assert g.info.kernel_path in (2, 5, 6) and g.info.tuned_plans >= 2
    h = pt.PT.from_problem(prob, kernel_path=2)
    for chunk in range(2):
        g.run(100, 1)
        o.run(100, 1)
        h.run(100, 1)
        assert_same(g, o, "sweep %d" % (100 * (chunk + 1)))
        assert np.array_equal(g.read_state(), h.read_state())
