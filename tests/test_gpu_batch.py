"""Batched persistent launch (pt_batch_*): every request gets exactly the bits it gets
alone (oracle and pt_create + pt_run), whatever the cluster size and whether its chains
stay resident in shared memory or stream through it."""
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


def _mixed_problems(n_sweeps):
    """Small requests of uneven shape: both neighbour classes, P 8..64, R 1..20, several swap cadences."""
    rng = np.random.default_rng(7)
    out = []
    specs = [("regular", dict(n=16, degree=3), 32, 16, 1), ("chimera", dict(rows=2, cols=2), 16, 5, 1),
             ("regular", dict(n=10, degree=3), 8, 3, 2), ("chimera", dict(rows=1, cols=3), 64, 7, 3),
             ("regular", dict(n=40, degree=3), 64, 20, 1), ("regular", dict(n=12, degree=3), 24, 1, 1),
             ("chimera", dict(rows=3, cols=2), 32, 2, 0), ("regular", dict(n=8, degree=3), 16, 9, 1)]
    for k, (graph, kw, P, R, sps) in enumerate(specs):
        prob = instances.make_problem(graph, rng, P=P, R=R, n_sweeps=n_sweeps, sweeps_per_swap=sps,
                                      seed=instances.philox_seed(900 + k), ladder="geometric", g0=0.1, g1=3.0,
                                      T=0.3, **kw)
        out.append(prob)
    return out


def _same(a_state, a_obs, b_state, b_obs, where):
    assert np.array_equal(a_state, b_state), where
    for key in b_obs:
        assert np.array_equal(np.asarray(a_obs[key]), np.asarray(b_obs[key])), (where, key)


def test_mixed_batch_matches_oracle_over_two_runs():
    probs = _mixed_problems(60)
    b = pt.Batch(probs)
    orcs = [Oracle.from_problem(p, threads=THREADS) for p in probs]
    for run in range(2):
        b.run()
        for k, (p, o) in enumerate(zip(probs, orcs)):
            o.run(p.n_sweeps, p.sweeps_per_swap)
            _same(b.read_state(k), b.obs(k), o.read_state(), o.obs(), "run %d request %d" % (run, k))


@pytest.mark.parametrize("cluster", [1, 2, 8])
def test_cluster_size_does_not_change_bits(cluster):
    probs = _mixed_problems(40)
    ref = pt.Batch(probs, cluster_size=4)
    alt = pt.Batch(probs, cluster_size=cluster)
    ref.run()
    alt.run()
    for k in range(len(probs)):
        _same(alt.read_state(k), alt.obs(k), ref.read_state(k), ref.obs(k), "cluster %d request %d" % (cluster, k))


def test_autotuned_layout_and_graph_replays_keep_the_bits():
    """cluster_size 0: pt_batch_create times each layout on a short run, resets the state and
    keeps the fastest; later runs replay one captured CUDA graph. Three runs, every request
    against the oracle and against a fixed layout."""
    probs = _mixed_problems(30)
    tuned = pt.Batch(probs)
    info = tuned.info()
    assert info.tuned_layouts >= 2 and info.cluster in (1, 2, 4, 8)
    fixed = pt.Batch(probs, cluster_size=2)
    assert fixed.info().tuned_layouts == 0
    orcs = [Oracle.from_problem(p, threads=THREADS) for p in probs]
    for run in range(3):
        tuned.run()
        fixed.run()
        for k, (p, o) in enumerate(zip(probs, orcs)):
            o.run(p.n_sweeps, p.sweeps_per_swap)
            _same(tuned.read_state(k), tuned.obs(k), o.read_state(), o.obs(), "tuned run %d request %d" % (run, k))
            _same(fixed.read_state(k), fixed.obs(k), o.read_state(), o.obs(), "fixed run %d request %d" % (run, k))
    assert tuned.info().graph == 1 and fixed.info().graph == 1


def test_run_recorded_into_a_callers_graph():
    """pt_batch_run on a stream under capture records the launch into the caller's graph;
    each replay is one more run, counters included."""
    torch = pytest.importorskip("torch")
    probs = _mixed_problems(20)
    stream = torch.cuda.Stream()
    b = pt.Batch(probs, cluster_size=2, stream=stream.cuda_stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.run()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for k, p in enumerate(probs):
        o = Oracle.from_problem(p, threads=THREADS)
        o.run(p.n_sweeps, p.sweeps_per_swap)
        o.run(p.n_sweeps, p.sweeps_per_swap)
        _same(b.read_state(k), b.obs(k), o.read_state(), o.obs(), "request %d" % k)


def test_batch_requests_equal_single_problem_runs():
    """A slice of the 512-request workload (uneven N, P, R): batched == one pt_run per request."""
    probs = instances.batch_problems(count=24, index=3, n_sweeps=30)
    b = pt.Batch(probs)
    b.run()
    for k, p in enumerate(probs):
        g = pt.PT.from_problem(p)
        g.run(p.n_sweeps, p.sweeps_per_swap)
        _same(b.read_state(k), b.obs(k), g.read_state(), g.obs(), "request %d" % k)
        g.close()


def test_large_chains_stream_through_shared_memory():
    """N=1024, P=128: a chain is 128 KiB, so a CTA sweeps its chains one after another out of
    global memory; the bits still match the oracle."""
    rng = np.random.default_rng(11)
    big = instances.make_problem("regular", rng, n=1024, degree=3, P=128, R=6, n_sweeps=12, sweeps_per_swap=1,
                                 seed=instances.philox_seed(77), ladder="geometric", g0=0.05, g1=4.0, T=0.02)
    small = instances.make_problem("chimera", rng, rows=4, cols=4, P=32, R=12, n_sweeps=12, sweeps_per_swap=1,
                                   seed=instances.philox_seed(78))
    probs = [big, small]
    b = pt.Batch(probs, cluster_size=2)
    b.run()
    for k, p in enumerate(probs):
        o = Oracle.from_problem(p, threads=THREADS)
        o.run(p.n_sweeps, p.sweeps_per_swap)
        _same(b.read_state(k), b.obs(k), o.read_state(), o.obs(), "request %d" % k)


def test_batch_rejects_unsupported_requests():
    rng = np.random.default_rng(1)
    odd_p = instances.make_problem("regular", rng, n=8, degree=3, P=6, R=2, n_sweeps=5)
    with pytest.raises(pt.PTError) as e:
        pt.Batch([odd_p])
    assert e.value.code == pt.PT_EINVAL


def test_batch_reports_the_first_unsupported_request_in_order():
    """Requests are prepared on several host threads; the error still names the first bad
    request by index, whichever thread met it."""
    rng = np.random.default_rng(2)
    probs = instances.batch_problems(count=96, index=3, n_sweeps=2)
    for k in (41, 77):
        probs[k] = instances.make_problem("regular", rng, n=8, degree=3, P=6, R=2, n_sweeps=2)
    with pytest.raises(pt.PTError) as e:
        pt.Batch(probs)
    assert e.value.code == pt.PT_EINVAL
    assert "request 41:" in str(e.value)


def _energy_and_trotter(prob, state):
    """E (summed over copies) and M of every rung of a rung-ordered state, recomputed."""
    s = state.astype(np.int64)  # [R, N, P]
    E = np.einsum("rep,e->r", s[:, prob.ei, :] * s[:, prob.ej, :], np.asarray(prob.J, np.int64))
    E += np.einsum("rip,i->r", s, np.asarray(prob.h, np.int64))
    M = (s * np.roll(s, -1, axis=2)).sum(axis=(1, 2))
    return E, M


def test_full_batched_workload_sampled_requests_and_invariants():
    """The bench's batched workload at full size and launch configuration (512 requests of
    the size mix, 1000 sweeps each, autotuned layout, graph replay): the smallest, a median
    and the largest request against the oracle bit for bit, and for every request E and M
    recomputed from its final state equal the accumulated values and the counters add up."""
    probs = instances.batch_problems(count=512, index=1, n_sweeps=1000)
    b = pt.Batch(probs)
    b.run()
    b.sync()
    work = [p.attempts_per_sweep * p.n_sweeps for p in probs]
    order = np.argsort(work, kind="stable")
    for k in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        o = Oracle.from_problem(probs[k], threads=THREADS)
        o.run(probs[k].n_sweeps, probs[k].sweeps_per_swap)
        _same(b.read_state(k), b.obs(k), o.read_state(), o.obs(), "request %d" % k)
    for k, p in enumerate(probs):
        ob = b.obs(k)
        E, M = _energy_and_trotter(p, b.read_state(k))
        assert np.array_equal(E, np.asarray(ob["E"])) and np.array_equal(M, np.asarray(ob["M"])), k
        assert ob["t"] == p.n_sweeps and ob["q"] == p.n_sweeps // p.sweeps_per_swap, k
        assert np.all(np.asarray(ob["n_meas"]) == p.n_sweeps), k
        assert np.all(np.asarray(ob["swap_acc"]) <= np.asarray(ob["swap_att"])), k
        assert sorted(np.asarray(ob["replica_at"]).tolist()) == list(range(p.R)), k
