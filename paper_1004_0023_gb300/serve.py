"""Serving driver: replays a Poisson arrival trace of PT-QMC requests.

Two modes on the same trace:
  batched -- the continuous-batching server of the C library (pt_server_*). In its default
             (streamed) mode each request is admitted as soon as a slot, arena room and the
             SMs its chains need are free, and launched at once with all of its sweeps on a
             stream of a pool, so requests that arrive while others run overlap with them on
             the device; a backlog starts together in one persistent batched launch, whose
             members complete on their own. (Stepped mode instead advances every admitted
             request by a quantum of sweeps per launch.)
  plain   -- one request at a time, first come first served, each with its own
             pt_create + pt_run + read (one problem per launch).
Latency = completion time - arrival time (host wall clock), where a request completes once
its final state and statistics have been read back to the host in both modes; throughput =
spin-flip attempts of the completed requests / wall time from the first arrival to the last
completion.
"""
from __future__ import annotations

import time

import numpy as np

from . import instances, pt


def poisson_trace(rate: float, duration: float, seed: int = 1, sweep_range=(500, 5000), count_cap=None):
    """Arrival times of a Poisson process and one request per arrival (sizes as the batched workload)."""
    rng = np.random.default_rng(seed)
    times = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration or (count_cap is not None and len(times) >= count_cap):
            break
        times.append(t)
    probs = instances.batch_problems(count=len(times), index=seed, n_sweeps=1)
    for p in probs:
        p.n_sweeps = int(rng.integers(sweep_range[0], sweep_range[1] + 1))
    return list(zip(times, probs))


def _summary(lat, attempts, wall, extra, arrived=None):
    """Latency percentiles over the completed requests, and over every arrival with the
    requests still unfinished at the deadline counted as infinitely late (None when the
    percentile falls on one of them)."""
    lat = np.asarray(lat, np.float64)
    d = {"completed": int(lat.size), "attempts_per_s": attempts / wall if wall > 0 else 0.0, "wall_s": wall}
    if lat.size:
        d.update(p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                 mean_s=float(lat.mean()), max_s=float(lat.max()))
    if arrived is not None:
        unfinished = max(0, int(arrived) - int(lat.size))
        d["unfinished"] = unfinished
        if arrived:
            allv = np.concatenate([lat, np.full(unfinished, np.inf)])
            for q, key in ((50, "p50_all_s"), (99, "p99_all_s")):
                v = float(np.percentile(allv, q, method="higher"))
                d[key] = v if np.isfinite(v) else None
    d.update(extra)
    return d


def replay_batched(trace, quantum_sweeps=100, max_active=512, arena_bytes=0, cluster_size=0, stream=None,
                   deadline=None, stepped=False, packed_only=False, poll_s=0.0005):
    """Drive the continuous-batching server in real time; stop admitting new work after `deadline` s."""
    srv = pt.Server(arena_bytes=arena_bytes, max_active=max_active, quantum_sweeps=quantum_sweeps,
                    cluster_size=cluster_size, stream=stream, stepped=stepped, packed_only=packed_only)
    arrival = {}
    done_t = {}
    attempts = {}
    k = 0
    t0 = time.perf_counter()
    max_mix = 0
    while len(done_t) < len(trace):
        now = time.perf_counter() - t0
        if deadline is not None and now > deadline:
            break
        while k < len(trace) and trace[k][0] <= now:
            rid = srv.submit(trace[k][1])
            arrival[rid] = trace[k][0]
            attempts[rid] = trace[k][1].attempts_per_sweep * trace[k][1].n_sweeps
            k += 1
        info = srv.info()
        if info.active == 0 and info.queued == 0:
            if k < len(trace):
                time.sleep(max(0.0, min(trace[k][0] - now, 0.01)))
            continue
        max_mix = max(max_mix, info.active)
        finished = srv.step()
        for rid in finished:
            srv.result(rid)  # the final state and statistics, read as the plain arm reads them
            done_t[rid] = time.perf_counter() - t0
            srv.release(rid)
        if not finished and not stepped:
            time.sleep(poll_s)
    wall = (max(done_t.values()) if done_t else 0.0) - (trace[0][0] if trace else 0.0)
    lat = [done_t[r] - arrival[r] for r in done_t]
    info = srv.info()
    out = _summary(lat, sum(attempts[r] for r in done_t), wall,
                   {"mode": "stepped" if stepped else "streamed", "submitted": k, "max_active_seen": max_mix,
                    "steps": int(info.steps), "wide_steps": int(info.wide_steps),
                    "group_launches": int(info.group_launches), "kernel_launches": int(info.kernel_launches),
                    "quantum_sweeps": quantum_sweeps}, arrived=len(trace))
    srv.close()
    return out


def replay_plain(trace, stream=None, deadline=None):
    """One request at a time: pt_create + pt_run + read, in arrival order. Plan timing at
    create is off: a one-off request of 500-5000 sweeps would spend a large share of its run
    timing candidate plans for a shape it never sees again."""
    t0 = time.perf_counter()
    lat, att, launches = [], 0, 0
    k = 0
    for arr, prob in trace:
        now = time.perf_counter() - t0
        if deadline is not None and now > deadline:
            break
        if arr > now:
            time.sleep(arr - now)
        ctx = pt.PT.from_problem(prob, stream=stream, no_autotune=1)
        ctx.run(prob.n_sweeps, prob.sweeps_per_swap)
        ctx.read_state()
        ctx.obs()
        lat.append(time.perf_counter() - t0 - arr)  # the result is on the host; teardown follows
        launches += int(ctx.get_info().kernel_launches)
        ctx.close()
        att += prob.attempts_per_sweep * prob.n_sweeps
        k += 1
    wall = (time.perf_counter() - t0) - (trace[0][0] if trace else 0.0)
    return _summary(lat, att, wall, {"mode": "plain", "submitted": k, "kernel_launches": launches},
                    arrived=len(trace))
