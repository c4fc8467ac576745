"""Continuous batching (pt_server_*): requests submitted at different times share launches
with whatever else is on the device, and each result is the same as the request run alone
(pt_create + pt_run) and as the oracle."""
import os
import time

import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import instances, pt, serve

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _lib(libpt):
    return libpt


def _requests(count, seed, sweep_range):
    rng = np.random.default_rng(seed)
    probs = instances.batch_problems(count=count, index=seed, n_sweeps=1, n_range=(16, 96), r_range=(2, 12),
                                     p_choices=(8, 16, 32))
    for p in probs:
        p.n_sweeps = int(rng.integers(sweep_range[0], sweep_range[1] + 1))
        p.sweeps_per_swap = int(rng.integers(1, 4))
    return probs


def _same(a_state, a_obs, b_state, b_obs, where):
    assert np.array_equal(a_state, b_state), where
    for key in b_obs:
        assert np.array_equal(np.asarray(a_obs[key]), np.asarray(b_obs[key])), (where, key)


@pytest.mark.parametrize("arena_bytes,max_active,stepped,packed_only",
                         [(0, 512, False, False), (1 << 20, 3, False, False), (0, 512, True, False),
                          (0, 512, True, True), (1 << 20, 3, True, False)])
def test_results_are_the_same_alone_and_in_the_mix(arena_bytes, max_active, stepped, packed_only):
    """Requests arrive over several steps; a small arena / slot count forces queueing; every
    mode (streamed launches, stepped with a CTA per chain, stepped with chains packed on
    clusters) gives each request the bits it gets alone."""
    probs = _requests(14, 5, (20, 90))
    srv = pt.Server(arena_bytes=arena_bytes, max_active=max_active, quantum_sweeps=16, stepped=stepped,
                    packed_only=packed_only)
    pending = list(enumerate(probs))
    ids, results, mix = {}, {}, 0
    while len(results) < len(probs):
        for _ in range(3):  # a few new arrivals before every step
            if pending:
                k, p = pending.pop(0)
                ids[srv.submit(p)] = k
        mix = max(mix, srv.info().active)
        for rid in srv.step():
            results[ids[rid]] = srv.result(rid)
            srv.release(rid)
        mix = max(mix, srv.info().active)
    assert mix >= 2 or max_active < 2
    for k, p in enumerate(probs):
        alone = pt.PT.from_problem(p)
        alone.run(p.n_sweeps, p.sweeps_per_swap)
        _same(results[k][0], results[k][1], alone.read_state(), alone.obs(), "request %d vs alone" % k)
        alone.close()
    for k in (0, 7):
        o = Oracle.from_problem(probs[k], threads=THREADS)
        o.run(probs[k].n_sweeps, probs[k].sweeps_per_swap)
        _same(results[k][0], results[k][1], o.read_state(), o.obs(), "request %d vs oracle" % k)
    _drain(srv)
    info = srv.info()
    assert info.active == 0 and info.queued == 0 and info.arena_used == 0
    if packed_only or not stepped:
        assert info.wide_steps == 0
    else:
        assert info.wide_steps > 0
    srv.close()


def _drain(srv):
    """A group's shared block is freed at the first step after its launch ends."""
    for _ in range(2000):
        if srv.info().arena_used == 0:
            return
        srv.step()
        time.sleep(0.001)
    assert srv.info().arena_used == 0


def test_backlog_starts_as_one_batched_launch_with_the_same_bits():
    """Twenty requests submitted before the first step form a backlog: they start together
    in one persistent batched launch, and each result still equals the request run alone."""
    probs = _requests(20, 9, (30, 120))
    srv = pt.Server()
    ids = {srv.submit(p): k for k, p in enumerate(probs)}
    results = {}
    while len(results) < len(probs):
        for rid in srv.step():
            results[ids[rid]] = srv.result(rid)
            srv.release(rid)
    info = srv.info()
    assert info.group_launches >= 1
    assert info.active == 0 and info.queued == 0
    _drain(srv)
    for k, p in enumerate(probs):
        alone = pt.PT.from_problem(p)
        alone.run(p.n_sweeps, p.sweeps_per_swap)
        _same(results[k][0], results[k][1], alone.read_state(), alone.obs(), "request %d vs alone" % k)
        alone.close()
    srv.close()


def test_server_rejects_a_request_larger_than_its_arena():
    srv = pt.Server(arena_bytes=1 << 16, max_active=4, quantum_sweeps=8)
    rng = np.random.default_rng(3)
    huge = instances.make_problem("regular", rng, n=512, degree=3, P=64, R=16, n_sweeps=5)
    with pytest.raises(pt.PTError) as e:
        srv.submit(huge)
    assert e.value.code == pt.PT_ENOMEM
    srv.close()


def test_poisson_replay_batched_and_plain_complete_every_request():
    trace = [(0.002 * i, p) for i, p in enumerate(_requests(10, 11, (30, 60)))]
    b = serve.replay_batched(trace, quantum_sweeps=16)
    st = serve.replay_batched(trace, quantum_sweeps=16, stepped=True)
    p = serve.replay_plain(trace)
    for r in (b, st, p):
        assert r["completed"] == 10
        assert r["p99_s"] >= r["p50_s"] > 0


def test_members_of_a_batched_launch_complete_on_their_own():
    """Nine requests submitted together start in one batched launch: one long request and
    eight short ones. The short ones complete (flagged by the kernel) while the long one is
    still running, and every result equals the request run alone."""
    short = _requests(8, 21, (20, 40))
    rng = np.random.default_rng(5)
    long_req = instances.make_problem("regular", rng, n=96, degree=3, P=32, R=12, n_sweeps=60000,
                                      seed=instances.philox_seed(77), ladder="geometric", g0=0.1, g1=3.0, T=0.2)
    probs = [long_req] + short
    srv = pt.Server()
    ids = {srv.submit(p): k for k, p in enumerate(probs)}
    order, results = [], {}
    while len(results) < len(probs):
        for rid in srv.step():
            k = ids[rid]
            order.append((k, srv.info().active))
            results[k] = srv.result(rid)
            srv.release(rid)
    assert srv.info().group_launches >= 1
    # the eight short requests came back first, each while the long one was still active
    assert [k for k, _ in order[:8]] != [] and 0 not in [k for k, _ in order[:8]]
    assert all(active >= 1 for _, active in order[:8])
    _drain(srv)
    for k, p in enumerate(probs):
        alone = pt.PT.from_problem(p)
        alone.run(p.n_sweeps, p.sweeps_per_swap)
        _same(results[k][0], results[k][1], alone.read_state(), alone.obs(), "request %d vs alone" % k)
        alone.close()
    srv.close()


def test_backlog_on_device_memory_that_held_other_data():
    """A server's arena is fresh device memory that may hold anything an earlier user left
    (here: small integers, like the completion tokens of an earlier server's batched
    launches). Long requests first occupy every stream of the server's pool, so that the
    backlog launched next waits behind one of them, zeroing of its flags included. Each
    member must still complete only once the kernel has written it back: the flags are read
    only after the launch's own zeroing has run, and tokens never repeat in a process. Every
    result equals the request run alone."""
    torch = pytest.importorskip("torch")
    arena = 256 << 20
    for round_ in range(2):
        junk = (torch.arange(arena // 4, dtype=torch.int32, device="cuda") % 64) + 1
        torch.cuda.synchronize()
        del junk
        torch.cuda.empty_cache()  # give the memory back, so the arena below can reuse it
        busy = _requests(16, 50 + round_, (20000, 30000))
        backlog = _requests(20, 40 + round_, (30, 120))
        probs = busy + backlog
        srv = pt.Server(arena_bytes=arena)
        ids, results = {}, {}
        for k, p in enumerate(busy):  # one at a time: each starts on its own launch and stream
            ids[srv.submit(p)] = k
            for rid in srv.step():
                results[ids[rid]] = srv.result(rid)
                srv.release(rid)
        for k, p in enumerate(backlog):
            ids[srv.submit(p)] = len(busy) + k
        while len(results) < len(probs):
            for rid in srv.step():
                results[ids[rid]] = srv.result(rid)
                srv.release(rid)
        assert srv.info().group_launches >= 1
        _drain(srv)
        srv.close()
        for k, p in enumerate(probs):
            alone = pt.PT.from_problem(p)
            alone.run(p.n_sweeps, p.sweeps_per_swap)
            _same(results[k][0], results[k][1], alone.read_state(), alone.obs(), "round %d request %d" % (round_, k))
            alone.close()
