#!/usr/bin/env python
"""Spin-flip attempts/s of the PT-QMC hot path (Metropolis sweeps + parity swaps) on GB300.

One step = one pass of the whole hot path over the workload: n_sweeps sweeps of every chain
with one swap pass after each sweep, on the state resident in HBM (the chain continues
from step to step, as a Markov chain does). Default workload: random 3-regular N=256,
P=64 Trotter copies, R=64 rungs (geometric Gamma 0.05..4.0 at T=0.02), 2000 sweeps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Under torchrun each rank runs its own independent problem (different seed) on its own GPU:
the work partitions into independent problems, so there is no data-path collective. The
only collectives are the barriers around each timed region and the max over ranks of its
time (with the sum of the units): the device-timed value, the end-to-end value and the
batched values are all whole-job figures. The serving replay runs on rank 0 alone.

--impl reference times the CPU oracle (the plain C implementation the tests compare against)
on this machine's host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "spin-flip attempts/s"
# Algorithmic integer lane-instructions per attempt, the work the method itself needs:
# 1/4 of a Philox4x32-10 call (10 rounds x (2 wide multiplies + 2 three-input XORs)) = 10,
# local field d multiply-adds, L = s*f (1), m = s*(s- + s+) (2), table index (2),
# acceptance compare (2), flip select (1), E/M/count updates (3).
def alg_instr_per_attempt(degree: int) -> int:
    return 10 + degree + 1 + 2 + 2 + 2 + 1 + 3


KERNEL_NAMES = {1: "sweep_kernel (byte-wise)", 2: "sweep_packed_kernel (int8, inline Philox)",
                3: "sweep_packed_kernel (int8, producer warps)", 4: "sweep_packed_kernel (bit-packed)",
                5: "sweep_split_kernel (int8, producer warps, each chain on a 2-CTA cluster)",
                6: "sweep_split_kernel (int8, inline Philox, each chain on a 2-CTA cluster)"}

# DRAM bytes (read + write) per launch of the sweep kernel, from one ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum: (workload, kernel path, sweeps per launch)
# -> bytes. Must be retaken (or removed) whenever that kernel changes.
MEASURED_TRAFFIC = {("regular3_n256_p64_r64", 2, 1000): (1648384 + 1893632) // 2,
                    ("chimera16_n2048_p128_r96", 4, 500): (26632448 + 11264 + 27145472) // 2}
# The same for the batched launch: (requests, sweeps each) -> DRAM bytes per launch.
MEASURED_BATCH_TRAFFIC = {(512, 1000): 1298192722688 + 1345140493056}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="regular3_n256_p64_r64")
    ap.add_argument("--sweeps", type=int, default=0, help="override sweeps per step (profiling runs)")
    ap.add_argument("--kernel-path", type=int, default=0,
                    help="force the main context's kernel path (profiling runs; 0 = autotuned at create)")
    ap.add_argument("--threads-per-block", type=int, default=0, help="force its block size (with --kernel-path)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-sweeps", type=int, default=1000)
    ap.add_argument("--batch-cluster", type=int, default=0, help="CTAs per cluster (0 = autotuned at create)")
    ap.add_argument("--serving-seconds", type=float, default=10.0)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--reference-budget-s", type=float, default=0.0,
                    help="--impl reference: seconds of oracle work per step (0 = fit the run in ~2.5 min)")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- distributed
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_timing(local_seconds: float, local_units: float, world: int, device=None):
    """Max of the timed region and sum of the units over ranks (weak scaling)."""
    if world == 1:
        return local_seconds, local_units
    import torch
    import torch.distributed as dist

    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "sm_min_mhz": min(sm) if sm else None, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1004_0023_gb300 import build as pbuild
    from paper_1004_0023_gb300 import instances, pt

    torch.cuda.set_device(local_rank)
    if rank == 0:
        pbuild.build()
    barrier(world)
    prob = instances.workload(args.workload, 1 + rank)
    if args.sweeps > 0:
        prob.n_sweeps = args.sweeps
    attempts_step = prob.attempts_per_sweep * prob.n_sweeps
    degree = int(np.bincount(np.concatenate([prob.ei, prob.ej]), minlength=prob.n).max())
    # a dedicated stream: the library launches on it and the CUDA events are recorded on it
    stream = torch.cuda.Stream()
    assert stream.cuda_stream != 0
    ctx = pt.PT.from_problem(prob, stream=stream.cuda_stream, kernel_path=args.kernel_path,
                             threads_per_block=args.threads_per_block)
    info = ctx.info

    def step():
        ctx.run(prob.n_sweeps, prob.sweeps_per_swap)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    torch.cuda.synchronize()

    # L2 (129 MB) is flushed between timed steps by writing a 512 MB buffer outside the events
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    sampler = ClockSampler(local_rank)
    if rank == 0:
        sampler.start()
    launches0 = ctx.get_info().kernel_launches
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    ctx.sync()
    wall = time.perf_counter() - wall0
    barrier(world)
    launches = ctx.get_info().kernel_launches - launches0
    clocks = sampler.stop() if rank == 0 else None
    step_ms = [a.elapsed_time(b) for a, b in times]
    local_s = sum(step_ms) / 1e3
    max_s, units = reduce_timing(local_s, float(attempts_step * args.steps), world,
                                 device=torch.device("cuda", local_rank))
    value = units / max_s

    # roofline of the dominant kernel (the sweep kernel; swaps run inside it)
    launches_per_step = launches / args.steps
    per_launch_s = (local_s / args.steps) / max(launches_per_step, 1)
    ialg = alg_instr_per_attempt(degree)
    achieved = ialg * attempts_step / (local_s / args.steps) / 1e12  # Tinstr/s
    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = n_sm * 128 * sm_max * 1e6 / 1e12

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, prob, pt, torch, world, torch.device("cuda", local_rank))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, budget_s=12.0)

    ctx.close()
    batched = None
    if not args.no_batched:
        batched = run_batched(args, pt, instances, torch, n_sm, sm_max, rank, world,
                              torch.device("cuda", local_rank))
    serving = None
    if not args.no_serving and rank == 0:
        serving = run_serving(args, torch, batched, local_rank)
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8/int32 (integer-exact)", "data": "synthetic",
        "config": {"workload": args.workload, "n": prob.n, "P": prob.P, "R": prob.R, "sweeps_per_step": prob.n_sweeps,
                   "sweeps_per_swap": prob.sweeps_per_swap, "degree": degree, "attempts_per_step": attempts_step,
                   "graph": "random 3-regular" if "regular" in args.workload else "K4,4 cell lattice",
                   "l2": "flushed between timed steps (512 MB write outside the events)",
                   "parallelism": "one independent problem per GPU" if world > 1 else "single GPU",
                   "threads_per_block": info.threads_per_block, "levels_per_sweep": info.n_levels,
                   "cooperative_swaps": bool(info.cooperative), "kernel_path": int(info.kernel_path),
                   "plans_timed_at_create": int(info.tuned_plans)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
                     "frac": achieved / peak,
                     "traffic": MEASURED_TRAFFIC.get((args.workload, int(info.kernel_path),
                                                      int(round(prob.n_sweeps / max(launches_per_step, 1))))),
                     "traffic_unit": "DRAM bytes per launch (ncu)",
                     "basis": "%d algorithmic integer lane-instructions per attempt; peak = %d SMs x 128 lanes x %.0f MHz"
                              % (ialg, n_sm, sm_max),
                     "kernel": KERNEL_NAMES.get(int(info.kernel_path), "sweep kernel"),
                     "launch_ms": per_launch_s * 1e3},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "batched": batched,
        "serving": serving,
    }


def run_batched(args, pt, instances, torch, n_sm, sm_max, rank=0, world=1, device=None):
    """Many independent requests in one persistent launch vs one pt_run per request.

    Workload: `batch_count` requests, N ~ U{32..1024} (3-regular or K4,4 cells), P ~ U{32,64,128},
    R ~ U{16..128}, `batch_sweeps` sweeps each, a swap pass after every sweep. With several
    ranks each runs its own request set; both values are the attempts of all ranks over the
    slowest rank's device time."""
    probs = instances.batch_problems(count=args.batch_count, index=1 + rank, n_sweeps=args.batch_sweeps)
    attempts = sum(p.attempts_per_sweep * p.n_sweeps for p in probs)
    stream = torch.cuda.Stream()
    t_create = time.perf_counter()
    b = pt.Batch(probs, cluster_size=args.batch_cluster, stream=stream.cuda_stream)  # 0: autotuned at create
    create_s = time.perf_counter() - t_create
    info = b.info()
    b.run()
    b.sync()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run()
    e1.record(stream)
    b.sync()
    torch.cuda.synchronize()
    barrier(world)
    local_ms = e0.elapsed_time(e1)
    max_s, all_attempts = reduce_timing(local_ms / 1e3, float(attempts), world, device=device)
    ms = max_s * 1e3
    b_graph = b.info().graph
    b.close()
    # plain path: every request through its own pt_create + pt_run, one after another
    ctxs = []
    for p in probs:
        ctxs.append(pt.PT.from_problem(p, stream=stream.cuda_stream))
    torch.cuda.synchronize()
    barrier(world)
    launches0 = sum(int(c.get_info().kernel_launches) for c in ctxs)  # create (and plan timing) excluded
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for c, p in zip(ctxs, probs):
        c.run(p.n_sweeps, p.sweeps_per_swap)
    p1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    plain_ms = reduce_timing(p0.elapsed_time(p1) / 1e3, float(attempts), world, device=device)[0] * 1e3
    plain_launches = sum(int(c.get_info().kernel_launches) for c in ctxs) - launches0
    for c in ctxs:
        c.close()
    value = all_attempts / (ms / 1e3)
    local_value = attempts / (local_ms / 1e3)  # this GPU's rate, against this GPU's peak
    deg = [max(np.bincount(np.concatenate([p.ei, p.ej]), minlength=p.n)) for p in probs]
    ialg = float(np.average([alg_instr_per_attempt(int(d)) for d in deg],
                            weights=[p.attempts_per_sweep * p.n_sweeps for p in probs]))
    peak = n_sm * 128 * sm_max * 1e6 / 1e12
    return {"workload": "%d requests, N~U{32..1024} 3-regular or K4,4 cells, P~U{32,64,128}, R~U{16..128}, "
                        "%d sweeps, swap pass after every sweep" % (args.batch_count, args.batch_sweeps),
            "value": value, "unit": "attempts/s", "ms": ms, "attempts": all_attempts,
            "plain_value": all_attempts / (plain_ms / 1e3), "plain_ms": plain_ms,
            "speedup_vs_plain": plain_ms / ms, "gpu_launches": 1, "plain_gpu_launches": plain_launches,
            "cluster": info.cluster, "n_clusters": info.n_clusters, "smem_bytes": int(info.smem_bytes),
            "group_widen": info.group_widen, "autotuned_layouts": info.tuned_layouts,
            "create_and_autotune_s": create_s, "graph_replay": bool(b_graph),
            "roofline": {"bound": "alu", "achieved": ialg * local_value / 1e12, "peak": peak, "unit": "Tinstr/s",
                         "frac": ialg * local_value / 1e12 / peak, "kernel": "batch_kernel",
                         "traffic": MEASURED_BATCH_TRAFFIC.get((args.batch_count, args.batch_sweeps)),
                         "traffic_unit": "DRAM bytes per launch (ncu)"}}


def run_serving(args, torch, batched, gpu_index=0):
    """Poisson arrivals of requests from the batched size distribution, 500..5000 sweeps each.

    The latency comparison at half capacity runs first, then the overload replay; SM clocks
    and throttle reasons are sampled during each."""
    from paper_1004_0023_gb300 import serve

    out = {"workload": "Poisson arrivals, sizes as the batched workload, sweeps~U{500..5000}, swap every sweep",
           "arrival_seconds": args.serving_seconds,
           "server": "continuous batching: requests admitted as slots and arena room free up, each launched on a "
                     "stream of a pool with one CTA per chain; plain = one request at a time, pt_create + pt_run"}
    stream = torch.cuda.Stream()
    trace = serve.poisson_trace(args.serving_rate, args.serving_seconds, seed=2)
    # a rate the batched server sustains (half its measured batched capacity), both modes
    if batched:
        mean_work = np.mean([p.attempts_per_sweep * p.n_sweeps for _, p in trace]) if trace else 1.0
        rate = max(1.0, 0.5 * batched["value"] / mean_work)
        trace2 = serve.poisson_trace(rate, args.serving_seconds, seed=3)
        sampler = ClockSampler(gpu_index)
        sampler.start()
        b = serve.replay_batched(trace2, stream=stream.cuda_stream, deadline=args.serving_seconds + 30.0)
        p = serve.replay_plain(trace2, stream=stream.cuda_stream, deadline=args.serving_seconds + 30.0)
        clocks = sampler.stop()
        for r in (b, p):
            r["rate_per_s"] = rate
            r["arrived"] = len(trace2)
        out["at_half_capacity"] = {"server": b, "plain": p, "clocks": clocks}
    offered = sum(p.attempts_per_sweep * p.n_sweeps for _, p in trace) / max(args.serving_seconds, 1e-9)
    sampler = ClockSampler(gpu_index)
    sampler.start()
    res = serve.replay_batched(trace, stream=stream.cuda_stream, deadline=args.serving_seconds + 30.0)
    res["clocks"] = sampler.stop()
    res["rate_per_s"] = args.serving_rate
    res["offered_attempts_per_s"] = offered
    res["arrived"] = len(trace)
    out["at_configured_rate"] = res
    return out


def run_e2e(args, prob, pt, torch, world=1, device=None):
    """Create from pinned host arrays, run, read state and statistics back, destroy.

    With several ranks each runs its own problem; the value is the units of all ranks over the
    slowest rank's time, like the device-timed value."""
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
    ei, ej, J, h = pin(prob.ei), pin(prob.ej), pin(prob.J), pin(prob.h)
    out = torch.empty((prob.R, prob.n, prob.P), dtype=torch.int8).pin_memory().numpy()
    res = {}

    def once():
        ctx = pt.PT(prob.n, ei, ej, J, h, prob.P, prob.T, prob.gamma, prob.seed)
        ctx.run(prob.n_sweeps, prob.sweeps_per_swap)
        ctx.read_state(out)
        ob = ctx.obs()
        res["h2d"] = ctx.get_info().h2d_bytes
        ctx.close()
        return ob

    for _ in range(max(1, min(args.warmup, 2))):
        once()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    n = max(1, min(args.steps, 5))
    for _ in range(n):
        once()
    torch.cuda.synchronize()
    local_s = time.perf_counter() - t0
    barrier(world)
    max_s, units = reduce_timing(local_s, float(prob.attempts_per_sweep * prob.n_sweeps * n), world, device=device)
    dt = max_s / n
    d2h = prob.R * prob.n * prob.P + prob.R * 8 * 8 + 2 * (prob.R - 1) * 8 + prob.R * 4
    return {"value": units / max_s, "unit": "attempts/s",
            "h2d_bytes_per_step": int(res["h2d"]), "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3,
            "what": "pt_create from pinned host arrays + pt_run + pt_read_state + pt_read_observables + pt_destroy"}


# ----------------------------------------------------------------------------- CPU oracle
def cpu_baseline(prob, budget_s=12.0, threads=None):
    """The CPU oracle as it stands, on the host cores, over a bounded sample of sweeps."""
    from oracle import Oracle
    from oracle import oracle as orc

    orc.build()
    threads = threads or os.cpu_count() or 1
    o = Oracle.from_problem(prob, threads=threads)
    t0 = time.perf_counter()
    o.run(2, prob.sweeps_per_swap)
    probe = max(time.perf_counter() - t0, 1e-6) / 2
    # the chain continues past one step's sweeps until the time budget is spent
    n = int(max(2, min(100 * max(prob.n_sweeps, 1), budget_s / probe)))
    t0 = time.perf_counter()
    o.run(n, prob.sweeps_per_swap)
    dt = time.perf_counter() - t0
    o.close()
    return {"value": prob.attempts_per_sweep * n / dt, "unit": "attempts/s", "cores": threads, "kind": "oracle",
            "sample": "%d sweeps (+ swap passes; %.2f steps of %d sweeps) of the same problem, one continuous "
                      "chain run, OpenMP over chains, %.1f s" % (n, n / max(prob.n_sweeps, 1), prob.n_sweeps, dt)}


def run_reference(args, rank, world):
    from paper_1004_0023_gb300 import instances

    if rank != 0:
        return None
    prob = instances.workload(args.workload, 1)
    threads = os.cpu_count() or 1
    per_step_budget = args.reference_budget_s or max(1.0, min(20.0, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        cpu_baseline(prob, budget_s=per_step_budget / 4, threads=threads)
    vals, t_total = [], 0.0
    for _ in range(args.steps):
        r = cpu_baseline(prob, budget_s=per_step_budget, threads=threads)
        vals.append(r["value"])
        t_total += prob.attempts_per_sweep / r["value"]
    value = float(np.mean(vals))
    return {
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * prob.attempts_per_sweep * prob.n_sweeps / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8/int32 (integer-exact)",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "n": prob.n, "P": prob.P, "R": prob.R, "sweeps_per_step": prob.n_sweeps,
                   "sweeps_per_swap": prob.sweeps_per_swap},
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": threads, "kind": "oracle",
                         "sample": "each step: a bounded number of sweeps (~%.0f s) of the workload" % per_step_budget},
        "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    args = parse_args(argv)
    rank, world, local_rank = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
