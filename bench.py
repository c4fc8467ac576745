#!/usr/bin/env python
"""Spin-flip attempts/s of the PT-QMC hot path (Metropolis sweeps + parity swaps) on GB300.

Headline (the default workload, "batched"): 512 independent requests in one persistent,
graph-captured launch -- N ~ U{32..1024} on random 3-regular graphs or K4,4 cell lattices,
P ~ U{32,64,128}, R ~ U{16..128}, 1000 sweeps each with a swap pass after every sweep. One
step = one such launch over every request (the chains continue from step to step, as a
Markov chain does); its state (about 1.45 GB of chains) is larger than L2. Beside it:
  - the same requests through the plain path, one pt_create + pt_run each (plain_value);
  - e2e: pt_batch_create from host arrays + pt_batch_run + every request's state and
    statistics read back + pt_batch_destroy, on the wall clock;
  - plain_configs: the single-problem workloads (N=16 P=32 R=16; N=256 P=64 R=64; the
    N=2048 K4,4 lattice, P=128 R=96, bit-packed; classical P=1 N=256 R=64), each timed on
    the device with its roofline and a CPU-oracle baseline;
  - serving: Poisson arrivals replayed against the continuous-batching server and against a
    plain one-request-at-a-time server, over a sweep of arrival rates.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Under torchrun each rank runs its own independent request set (seed 1 + rank) on its own
GPU: the work partitions into independent problems, so there is no data-path collective.
The only collectives are the barriers around each timed region and the max over ranks of
its time (with the sum of the units). The serving replay runs on rank 0 alone.

--impl reference times the CPU oracle (the plain C implementation the tests compare against)
on this machine's host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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
PLAIN_CONFIGS = ("regular3_n16_p32_r16", "regular3_n256_p64_r64", "chimera16_n2048_p128_r96",
                 "classical_regular3_n256_r64")


def alg_instr_per_attempt(degree: int) -> int:
    """Algorithmic integer lane-instructions per attempt, counted as the method needs them:
    reads of d neighbour spins, d packed (index, J) words, h, the 2 Trotter neighbours and 1
    threshold entry (2d + 4); the conditional spin write (1); 1/4 of a Philox4x32-10 call
    (10 rounds x (2 wide multiplies + 2 three-input XORs) over 4 copies: 10); d multiply-adds
    of the field; and about 5 for the index, compare and select: 22 + 3d, i.e. 31 for
    degree 3 and 40 for degree 6."""
    return 22 + 3 * degree


def alg_instr_arith_only(degree: int) -> int:
    """The same without the loads and the store (arithmetic alone): Philox 10, field d,
    L = s f 1, m 2, table index 2, compare 2, flip 1, E/M/count 3: 21 + d."""
    return 21 + degree


KERNEL_NAMES = {1: "sweep_kernel (byte-wise)", 2: "sweep_packed_kernel (int8, inline Philox)",
                3: "sweep_packed_kernel (int8, producer warps)", 4: "sweep_packed_kernel (bit-packed)",
                5: "sweep_split_kernel (int8, producer warps, each chain on a 2-CTA cluster)",
                6: "sweep_split_kernel (int8, inline Philox, each chain on a 2-CTA cluster)",
                7: "batch_kernel (all chains of the problem packed on one cluster, swaps in shared memory)",
                8: "sweep_peer_kernel (int8, random words from a second CTA of each chain's cluster)",
                9: "sweep_cluster_kernel (int8, every chain's CTA in one cluster, swap mailboxes in shared memory)",
                10: "sweep_classical_kernel (P = 1, chains packed several to a CTA on one cluster)"}


# The sources each kernel is compiled from (its own file and the headers it includes).
KERNEL_SOURCES = {"sweep": ("pt_kernels.cu", "pt_device.cuh", "pt_internal.h"),
                  "batch": ("pt_batch.cu", "pt_device.cuh", "pt_internal.h")}


def kernel_source_hash(which: str) -> str:
    """First 16 hex digits of a SHA-256 over one kernel's sources (and include/pt.h): DRAM
    traffic figures below are reported only for the build they were measured on."""
    d = os.path.join(ROOT, "paper_1004_0023_gb300", "csrc")
    h = hashlib.sha256()
    for path in [os.path.join(d, f) for f in KERNEL_SOURCES[which]] + [os.path.join(ROOT, "include", "pt.h")]:
        with open(path, "rb") as fh:
            h.update(os.path.basename(path).encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the dominant
# kernel, from one ncu capture: (kernel, workload key) -> (source set, kernel_source_hash()
# of the build captured, bytes). A figure whose hash no longer matches is reported as null.
MEASURED_TRAFFIC: dict = {
    # one 1000-sweep launch of the N=256, P=64, R=64 plan (path 8, 384 threads): 1.67 MB read, 0 written
    ("sweep_peer_kernel (int8, random words from a second CTA of each chain's cluster)", "regular3_n256_p64_r64_2000"):
        ("sweep", "f982c437e1429c9c", 1646848),
    # one 500-sweep launch of the K4,4 lattice, bit-packed (path 4, 512 threads)
    ("sweep_packed_kernel (bit-packed)", "chimera16_n2048_p128_r96_500"): ("sweep", "f982c437e1429c9c", 26689280 + 4096),
    # one graph-replayed launch of the 512-request mix, 1000 sweeps each (clusters of 2, one
    # warp per chain): 1.286 TB read + 1.342 TB written, 1.85 B per attempt
    ("batch_kernel", "batched_512x1000"): ("batch", "5d28179cf3346bf2", 1285770739456 + 1342508638720),
}


def measured_traffic(kernel: str, key: str):
    ent = MEASURED_TRAFFIC.get((kernel, key))
    if ent is None:
        return None, "no ncu capture recorded for this kernel and workload"
    which, src, nbytes = ent
    if src != kernel_source_hash(which):
        return None, "stale: the kernel sources changed since the ncu capture (%s)" % src
    return nbytes, "ncu dram__bytes_read.sum + dram__bytes_write.sum, per launch"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="batched",
                    help="'batched' (the 512-request launch) or a single-problem workload name")
    ap.add_argument("--sweeps", type=int, default=0, help="override sweeps per step (profiling runs)")
    ap.add_argument("--kernel-path", type=int, default=0,
                    help="single-problem workload: force the kernel path (profiling runs; 0 = autotuned)")
    ap.add_argument("--threads-per-block", type=int, default=0, help="force its block size (with --kernel-path)")
    ap.add_argument("--cluster-size", type=int, default=0, help="with --kernel-path 7: CTAs of the one cluster")
    ap.add_argument("--group-threads", type=int, default=0, help="with --kernel-path 7: threads per chain group")
    ap.add_argument("--producer-threads", type=int, default=0,
                    help="with --kernel-path 3, 5 or 9: random-word producer threads per CTA")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain-compare", action="store_true", help="skip the one-pt_run-per-request comparison")
    ap.add_argument("--no-plain-configs", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-sweeps", type=int, default=1000)
    ap.add_argument("--batch-cluster", type=int, default=0, help="CTAs per cluster (0 = autotuned at create)")
    ap.add_argument("--plain-steps", type=int, default=5, help="timed steps of each single-problem sub-record")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="arrival window of the half-capacity comparison")
    ap.add_argument("--sweep-seconds", type=float, default=10.0, help="arrival window of each other rate")
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--overload-seconds", type=float, default=10.0)
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


def max_degree(prob) -> int:
    if prob.ei.size == 0:
        return 0
    return int(np.bincount(np.concatenate([prob.ei, prob.ej]), minlength=prob.n).max())


def issue_peak(n_sm: int, sm_mhz: float) -> float:
    """Integer issue roof in T lane-instructions/s: SMs x 4 schedulers x 32 lanes x clock."""
    return n_sm * 128 * sm_mhz * 1e6 / 1e12


def roofline(ialg: float, iarith: float, attempts_per_launch: float, launch_s: float, n_sm: int, sm_mhz: float,
             kernel: str, traffic_key: str):
    achieved = ialg * attempts_per_launch / launch_s / 1e12
    peak = issue_peak(n_sm, sm_mhz)
    traffic, note = measured_traffic(kernel, traffic_key)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tinstr/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_note": note,
            "basis": "%.1f algorithmic integer lane-instructions per attempt (22 + 3d, loads and store included); "
                     "peak = %d SMs x 128 lanes x %.0f MHz (of measured clock)" % (ialg, n_sm, sm_mhz),
            "frac_arith_only": iarith * attempts_per_launch / launch_s / 1e12 / peak,
            "arith_only_basis": "%.1f per attempt (21 + d, arithmetic without loads and store)" % iarith,
            "kernel": kernel, "launch_ms": launch_s * 1e3, "attempts_per_launch": attempts_per_launch}


# ----------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1004_0023_gb300 import build as pbuild
    from paper_1004_0023_gb300 import instances, pt

    torch.cuda.set_device(local_rank)
    if rank == 0:
        pbuild.build()
    barrier(world)
    device = torch.device("cuda", local_rank)
    n_sm = torch.cuda.get_device_properties(local_rank).multi_processor_count
    if args.workload == "batched":
        out = batched_headline(args, pt, instances, torch, n_sm, rank, world, local_rank, device)
    else:
        out = plain_headline(args, pt, instances, torch, n_sm, rank, world, local_rank, device)
    if not args.no_plain_configs and args.workload == "batched":
        sm_mhz = (out.get("clocks") or {}).get("sm_max_mhz") or 2070.0
        out["plain_configs"] = [plain_record(name, args, pt, instances, torch, n_sm, sm_mhz, rank, world, device)
                                for name in PLAIN_CONFIGS]
    if not args.no_serving and rank == 0 and args.workload == "batched":
        out["serving"] = run_serving(args, torch, out["value"] / max(world, 1), local_rank)
    return out if rank == 0 else None


def batched_headline(args, pt, instances, torch, n_sm, rank, world, local_rank, device):
    """The 512-request persistent launch: value, plain comparison, e2e, roofline, CPU baseline."""
    probs = instances.batch_problems(count=args.batch_count, index=1 + rank, n_sweeps=args.batch_sweeps)
    if args.sweeps > 0:
        for p in probs:
            p.n_sweeps = args.sweeps
    attempts = float(sum(p.attempts_per_sweep * p.n_sweeps for p in probs))
    weights = [p.attempts_per_sweep * p.n_sweeps for p in probs]
    degs = [max_degree(p) for p in probs]
    ialg = float(np.average([alg_instr_per_attempt(d) for d in degs], weights=weights))
    iarith = float(np.average([alg_instr_arith_only(d) for d in degs], weights=weights))
    stream = torch.cuda.Stream()
    t_create = time.perf_counter()
    b = pt.Batch(probs, cluster_size=args.batch_cluster, stream=stream.cuda_stream)  # 0: autotuned at create
    create_s = time.perf_counter() - t_create
    info = b.info()
    for _ in range(args.warmup):
        b.run()
    b.sync()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    if rank == 0:
        sampler.start()
    launches0 = b.info().kernel_launches
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    evs = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run()  # one graph replay: work-counter reset + the persistent launch
        e1.record(stream)
        evs.append((e0, e1))
    b.sync()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clocks = sampler.stop() if rank == 0 else None
    launches = int(b.info().kernel_launches - launches0)
    step_ms = [a.elapsed_time(c) for a, c in evs]
    local_s = sum(step_ms) / 1e3
    max_s, units = reduce_timing(local_s, attempts * args.steps, world, device=device)
    value = units / max_s
    graph = bool(b.info().graph)
    b.close()
    sm_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    launch_s = local_s / args.steps
    rf = roofline(ialg, iarith, attempts, launch_s, n_sm, sm_mhz, "batch_kernel",
                  "batched_%dx%d" % (args.batch_count, probs[0].n_sweeps))

    plain = None
    if not args.no_plain_compare:
        plain = plain_compare(probs, attempts, pt, torch, stream, world, device)
    e2e = None
    if not args.no_e2e:
        e2e = batched_e2e(args, probs, attempts, pt, torch, stream, world, device)
    cpu = cpu_mt = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_batch_sample(probs, budget_s=16.0)
        cpu_mt = cpu_batch_sample(probs, budget_s=8.0, kind="paper_mt")
    workload = ("%d requests, N~U{32..1024} random 3-regular or K4,4 cell lattice, P~U{32,64,128}, R~U{16..128}, "
                "J in {-2,-1,1,2}, h in {-1,0,1}, geometric Gamma 0.05..4.0 at T=0.02, %d sweeps each, swap pass "
                "after every sweep" % (args.batch_count, probs[0].n_sweeps))
    out = {
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int8/int32 (integer-exact)", "data": "synthetic",
        "config": {"workload": "batched_%dx%d" % (args.batch_count, probs[0].n_sweeps), "description": workload,
                   "requests": len(probs), "attempts_per_step": attempts,
                   "chain_bytes": int(sum(p.n * p.P * p.R for p in probs)),
                   "l2": "not flushed: the chains (%.2f GB) are larger than L2 and every step reads them"
                         % (sum(p.n * p.P * p.R for p in probs) / 1e9),
                   "parallelism": "one independent request set per GPU" if world > 1 else "single GPU",
                   "cluster": info.cluster, "n_clusters": info.n_clusters, "threads_per_block": info.threads_per_block,
                   "smem_bytes": int(info.smem_bytes), "group_widen": info.group_widen,
                   "layouts_timed_at_create": info.tuned_layouts, "create_and_autotune_s": create_s,
                   "graph_replay": graph},
        "step_ms": {"min": float(np.min(step_ms)), "median": float(np.median(step_ms)), "max": float(np.max(step_ms))},
        "roofline": rf,
        "cpu_baseline": cpu,
        "cpu_paper_mt": cpu_mt,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    if plain:
        out.update(plain)
        out["speedup_vs_plain"] = value / plain["plain_value"]
    return out


def plain_compare(probs, attempts, pt, torch, stream, world, device):
    """The same requests through the plain path: one pt_create (autotuned) + pt_run each,
    one after another on one stream. Create and plan timing are outside the events."""
    ctxs = [pt.PT.from_problem(p, stream=stream.cuda_stream) for p in probs]
    torch.cuda.synchronize()
    barrier(world)
    launches0 = sum(int(c.get_info().kernel_launches) for c in ctxs)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for c, p in zip(ctxs, probs):
        c.run(p.n_sweeps, p.sweeps_per_swap)
    p1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    max_s, units = reduce_timing(p0.elapsed_time(p1) / 1e3, attempts, world, device=device)
    launches = sum(int(c.get_info().kernel_launches) for c in ctxs) - launches0
    for c in ctxs:
        c.close()
    return {"plain_value": units / max_s, "plain_ms": max_s * 1e3, "plain_gpu_launches": int(launches),
            "plain_what": "one pt_create (plan autotuned, outside the timing) + pt_run per request, in sequence"}


def batched_e2e(args, probs, attempts, pt, torch, stream, world, device):
    """pt_batch_create from host arrays + pt_batch_run + every request's state (into pinned
    buffers) and statistics + pt_batch_destroy, on the wall clock. The layout the autotuner
    chose for this batch shape is remembered by the library, so these creates time nothing."""
    outs = [torch.empty((p.R, p.n, p.P), dtype=torch.int8).pin_memory().numpy() for p in probs]
    res = {}

    def once():
        bb = pt.Batch(probs, cluster_size=args.batch_cluster, stream=stream.cuda_stream)
        bb.run()
        for k in range(len(probs)):
            bb.read_state(k, outs[k])
            bb.obs(k)
        res["h2d"] = int(bb.info().h2d_bytes)
        res["tuned"] = int(bb.info().tuned_layouts)
        bb.close()

    once()
    torch.cuda.synchronize()
    barrier(world)
    n = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(n):
        once()
    torch.cuda.synchronize()
    local_s = time.perf_counter() - t0
    barrier(world)
    max_s, units = reduce_timing(local_s, attempts * n, world, device=device)
    d2h = sum(p.R * p.n * p.P + p.R * 8 * 8 + 2 * max(p.R - 1, 1) * 8 + p.R * 4 for p in probs)
    return {"value": units / max_s, "unit": "attempts/s", "h2d_bytes_per_step": res["h2d"],
            "d2h_bytes_per_step": int(d2h), "ms_per_step": max_s / n * 1e3, "steps": n,
            "layouts_timed_in_timed_creates": res["tuned"],
            "what": "pt_batch_create from host arrays + pt_batch_run + pt_batch_read_state (pinned) and "
                    "pt_batch_read_observables of every request + pt_batch_destroy"}


def plain_headline(args, pt, instances, torch, n_sm, rank, world, local_rank, device):
    """One single-problem workload as the headline (profiling runs)."""
    prob = instances.workload(args.workload, 1 + rank)
    if args.sweeps > 0:
        prob.n_sweeps = args.sweeps
    rec = plain_record(args.workload, args, pt, instances, torch, n_sm, None, rank, world, device, prob=prob,
                       steps=args.steps, warmup=args.warmup, kernel_path=args.kernel_path,
                       threads_per_block=args.threads_per_block, clocks=True, cluster_size=args.cluster_size,
                       group_threads=args.group_threads, producer_threads=args.producer_threads)
    out = {"metric": METRIC, "value": rec["value"], "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int8/int32 (integer-exact)", "data": "synthetic",
           "config": rec["config"], "roofline": rec["roofline"], "cpu_baseline": rec["cpu_baseline"],
           "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"], "e2e": None}
    if not args.no_e2e:
        out["e2e"] = plain_e2e(args, prob, pt, torch, world, device)
    return out


def plain_record(name, args, pt, instances, torch, n_sm, sm_mhz, rank, world, device, prob=None, steps=None,
                 warmup=2, kernel_path=0, threads_per_block=0, clocks=False, cluster_size=0, group_threads=0,
                 producer_threads=0):
    """A single-problem workload on the device: the autotuned plan, L2 flushed between
    timed steps, value, roofline and a CPU-oracle baseline."""
    prob = prob or instances.workload(name, 1 + rank)
    steps = steps or args.plain_steps
    stream = torch.cuda.Stream()
    ctx = pt.PT.from_problem(prob, stream=stream.cuda_stream, kernel_path=kernel_path,
                             threads_per_block=threads_per_block, cluster_size=cluster_size,
                             group_threads=group_threads, producer_threads=producer_threads)
    info = ctx.info
    for _ in range(warmup):
        ctx.run(prob.n_sweeps, prob.sweeps_per_swap)
    ctx.sync()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=device)
    sampler = ClockSampler(device.index or 0)
    if clocks and rank == 0:
        sampler.start()
    launches0 = ctx.get_info().kernel_launches
    torch.cuda.synchronize()
    barrier(world)
    evs = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)  # L2 (129 MB) flushed outside the events
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.run(prob.n_sweeps, prob.sweeps_per_swap)
        e1.record(stream)
        evs.append((e0, e1))
    ctx.sync()
    torch.cuda.synchronize()
    barrier(world)
    ck = sampler.stop() if (clocks and rank == 0) else None
    del flush
    launches = int(ctx.get_info().kernel_launches - launches0)
    step_ms = [a.elapsed_time(c) for a, c in evs]
    local_s = sum(step_ms) / 1e3
    attempts = float(prob.attempts_per_sweep * prob.n_sweeps)
    max_s, units = reduce_timing(local_s, attempts * steps, world, device=device)
    d = max_degree(prob)
    mhz = sm_mhz or (ck or {}).get("sm_max_mhz") or 2070.0
    per_launch = local_s / max(launches, 1)
    rf = roofline(alg_instr_per_attempt(d), alg_instr_arith_only(d), attempts * steps / max(launches, 1), per_launch,
                  n_sm, mhz, KERNEL_NAMES.get(int(info.kernel_path), "sweep kernel"),
                  "%s_%d" % (name, prob.n_sweeps))
    ctx.close()
    cpu = cpu_mt = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, budget_s=4.0 if not clocks else 12.0)
        cpu_mt = cpu_baseline(prob, budget_s=3.0, kind="paper_mt")
    return {"workload": name, "value": units / max_s, "unit": "attempts/s", "ms_per_step": float(np.mean(step_ms)),
            "steps": steps, "gpu_launches": launches, "clocks": ck,
            "config": {"workload": name, "n": prob.n, "P": prob.P, "R": prob.R, "degree": d,
                       "sweeps_per_step": prob.n_sweeps, "sweeps_per_swap": prob.sweeps_per_swap,
                       "attempts_per_step": attempts, "kernel_path": int(info.kernel_path),
                       "threads_per_block": int(info.threads_per_block), "levels_per_sweep": int(info.n_levels),
                       "cooperative_swaps": bool(info.cooperative), "plans_timed_at_create": int(info.tuned_plans),
                       "l2": "flushed between timed steps (512 MB write outside the events)"},
            "roofline": rf, "cpu_baseline": cpu, "cpu_paper_mt": cpu_mt}


def plain_e2e(args, prob, pt, torch, world=1, device=None):
    """Create from pinned host arrays, run, read state and statistics back, destroy."""
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
    d2h = prob.R * prob.n * prob.P + prob.R * 8 * 8 + 2 * (prob.R - 1) * 8 + prob.R * 4
    return {"value": units / max_s, "unit": "attempts/s", "h2d_bytes_per_step": int(res["h2d"]),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": max_s / n * 1e3,
            "what": "pt_create from pinned host arrays + pt_run + pt_read_state + pt_read_observables + pt_destroy"}


# ----------------------------------------------------------------------------- serving
def run_serving(args, torch, capacity, gpu_index=0):
    """Poisson arrivals of requests from the batched size distribution, 500..5000 sweeps each,
    against the continuous-batching server and a plain one-request-at-a-time server, at
    0.25, 0.5, 0.75, 1.0 and 1.5 x the measured batched capacity (at the trace's mean request
    size), then at the configured overload rate. SM clocks are sampled during each replay."""
    from paper_1004_0023_gb300 import serve

    out = {"workload": "Poisson arrivals, sizes as the batched workload, sweeps~U{500..5000}, swap every sweep",
           "server": "continuous batching: requests admitted as slots, arena room and SMs free up, each launched "
                     "on a pool stream with one CTA per chain; a backlog of 8 or more starts in one persistent "
                     "batched launch whose cluster size follows the free SMs",
           "plain": "one request at a time: pt_create + pt_run + read, first come first served",
           "latency": "completion (state and statistics read to the host) - arrival, both arms",
           "capacity_attempts_per_s": capacity}
    stream = torch.cuda.Stream()
    probe = serve.poisson_trace(50.0, 20.0, seed=2)
    mean_work = float(np.mean([p.attempts_per_sweep * p.n_sweeps for _, p in probe]))
    curve = []
    for k, frac in enumerate((0.25, 0.5, 0.75, 1.0, 1.5)):
        seconds = args.serving_seconds if frac == 0.5 else args.sweep_seconds
        rate = max(0.5, frac * capacity / mean_work)
        trace = serve.poisson_trace(rate, seconds, seed=10 + k)
        sampler = ClockSampler(gpu_index)
        sampler.start()
        b = serve.replay_batched(trace, stream=stream.cuda_stream, deadline=seconds + 15.0)
        p = serve.replay_plain(trace, stream=stream.cuda_stream, deadline=seconds + 5.0)
        clocks = sampler.stop()
        curve.append({"fraction_of_capacity": frac, "rate_per_s": rate, "arrival_seconds": seconds,
                      "arrived": len(trace), "server": b, "plain": p, "clocks": clocks})
    out["rate_sweep"] = curve
    trace = serve.poisson_trace(args.serving_rate, args.overload_seconds, seed=2)
    offered = sum(p.attempts_per_sweep * p.n_sweeps for _, p in trace) / max(args.overload_seconds, 1e-9)
    sampler = ClockSampler(gpu_index)
    sampler.start()
    # about 3x capacity: the queue drains for about twice the arrival window after it closes
    res = serve.replay_batched(trace, stream=stream.cuda_stream, deadline=args.overload_seconds + 50.0)
    res["clocks"] = sampler.stop()
    res.update(rate_per_s=args.serving_rate, arrival_seconds=args.overload_seconds, offered_attempts_per_s=offered,
               arrived=len(trace))
    out["at_configured_rate"] = res
    return out


# ----------------------------------------------------------------------------- CPU oracle
def cpu_baseline(prob, budget_s=12.0, threads=None, kind="oracle"):
    """A CPU implementation on the host cores over a bounded sample of sweeps: the oracle as it
    stands (kind "oracle"), or the paper's multi-threaded design (kind "paper_mt")."""
    threads = threads or os.cpu_count() or 1
    if kind == "oracle":
        from oracle import Oracle
        from oracle import oracle as orc

        orc.build()
        o = Oracle.from_problem(prob, threads=threads)
    else:
        from cpu_pt import CpuPT

        o = CpuPT.from_problem(prob, threads=threads)
    t0 = time.perf_counter()
    o.run(2, prob.sweeps_per_swap)
    probe = max(time.perf_counter() - t0, 1e-6) / 2
    # the chain continues past one step's sweeps until the time budget is spent
    n = int(max(2, min(100 * max(prob.n_sweeps, 1), budget_s / probe)))
    t0 = time.perf_counter()
    o.run(n, prob.sweeps_per_swap)
    dt = time.perf_counter() - t0
    o.close()
    how = "OpenMP over chains" if kind == "oracle" else "persistent threads, work pool hardest chain first"
    return {"value": prob.attempts_per_sweep * n / dt, "unit": "attempts/s", "cores": threads, "kind": kind,
            "sample": "%d sweeps (+ swap passes; %.2f steps of %d sweeps) of the same problem, one continuous "
                      "chain run, %s, %.1f s" % (n, n / max(prob.n_sweeps, 1), prob.n_sweeps, how, dt)}


def cpu_batch_sample(probs, budget_s=16.0, threads=None, picks=8, kind="oracle"):
    """A CPU implementation on a seeded sample of the batched mix: `picks` requests spread
    evenly over the mix (indices 0, count/picks, ...), each run for an equal share of the time
    budget. kind "oracle": the plain oracle (OpenMP over chains); "paper_mt": the paper's
    multi-threaded design (persistent threads, work pool hardest chain first, Sec. 4)."""
    threads = threads or os.cpu_count() or 1
    if kind == "oracle":
        from oracle import Oracle
        from oracle import oracle as orc

        orc.build()
        make = lambda p: Oracle.from_problem(p, threads=threads)  # noqa: E731
    else:
        from cpu_pt import CpuPT

        make = lambda p: CpuPT.from_problem(p, threads=threads)  # noqa: E731
    idx = [int(k * len(probs) / picks) for k in range(min(picks, len(probs)))]
    att, secs, sweeps = 0.0, 0.0, []
    for k in idx:
        p = probs[k]
        o = make(p)
        t0 = time.perf_counter()
        o.run(1, p.sweeps_per_swap)
        probe = max(time.perf_counter() - t0, 1e-6)
        n = int(max(1, min(p.n_sweeps, (budget_s / len(idx)) / probe)))
        t0 = time.perf_counter()
        o.run(n, p.sweeps_per_swap)
        secs += time.perf_counter() - t0
        att += float(p.attempts_per_sweep) * n
        sweeps.append(n)
        o.close()
    how = "OpenMP over chains" if kind == "oracle" else "persistent threads, work pool hardest chain first"
    return {"value": att / secs, "unit": "attempts/s", "cores": threads, "kind": kind,
            "sample": "requests %s of the %d-request mix, %s sweeps each (+ swap passes), %s, %.1f s of CPU time"
                      % (idx, len(probs), sweeps, how, secs)}


def run_reference(args, rank, world):
    from paper_1004_0023_gb300 import instances

    if rank != 0:
        return None
    threads = os.cpu_count() or 1
    per_step_budget = args.reference_budget_s or max(1.0, min(20.0, 150.0 / max(args.steps + args.warmup, 1)))
    if args.workload == "batched":
        probs = instances.batch_problems(count=args.batch_count, index=1, n_sweeps=args.batch_sweeps)
        attempts = float(sum(p.attempts_per_sweep * p.n_sweeps for p in probs))
        measure = lambda budget: cpu_batch_sample(probs, budget_s=budget, threads=threads)  # noqa: E731
        config = {"workload": "batched_%dx%d" % (args.batch_count, args.batch_sweeps), "requests": len(probs),
                  "attempts_per_step": attempts}
    else:
        prob = instances.workload(args.workload, 1)
        attempts = float(prob.attempts_per_sweep * prob.n_sweeps)
        measure = lambda budget: cpu_baseline(prob, budget_s=budget, threads=threads)  # noqa: E731
        config = {"workload": args.workload, "n": prob.n, "P": prob.P, "R": prob.R,
                  "sweeps_per_step": prob.n_sweeps, "sweeps_per_swap": prob.sweeps_per_swap}
    for _ in range(args.warmup):
        measure(per_step_budget / 4)
    vals = [measure(per_step_budget)["value"] for _ in range(args.steps)]
    value = float(np.mean(vals))
    return {
        "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * attempts / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8/int32 (integer-exact)",
        "data": "synthetic", "impl": "reference", "config": config,
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": threads, "kind": "oracle",
                         "sample": "each step: a bounded sample (~%.0f s of oracle time) of the workload"
                                   % per_step_budget},
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
