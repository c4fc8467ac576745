"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): the max-over-ranks timing
and the sum of units, the end-to-end and batched figures as whole-job values (with fake
device objects), and the reference arm printing one line from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed (r + 1) seconds for 10 (r + 1) units
    t, u = bench.reduce_timing(float(rank + 1), 10.0 * (rank + 1), world, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump([t, u], f)


def test_reduce_timing_takes_max_seconds_and_sum_of_units(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_reduce_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        with open(tmp_path / ("rank%d.json" % r)) as f:
            assert json.load(f) == [2.0, 30.0]


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    pytest.importorskip("torch.distributed")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "1", "--workload", "regular3_n16_p32_r16",
           "--reference-budget-s", "0.3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


class _FakeEvent:
    """Stands in for torch.cuda.Event: rank r's timed regions last 10 (r + 1) ms."""
    rank = 0

    def __init__(self, enable_timing=True):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 10.0 * (_FakeEvent.rank + 1)


class _FakeInfo:
    h2d_bytes = 100
    threads_per_block = 512
    kernel_launches = 0
    cluster = 2
    n_clusters = 76
    smem_bytes = 1
    group_widen = 0
    tuned_layouts = 1
    graph = 1


class _FakeCtx:
    def __init__(self, *a, **k):
        pass

    @classmethod
    def from_problem(cls, prob, **k):
        return cls()

    def run(self, *a):
        pass

    def read_state(self, out=None):
        pass

    def obs(self):
        return {}

    def get_info(self):
        return _FakeInfo()

    def close(self):
        pass


class _FakeBatch(_FakeCtx):
    def __init__(self, probs, **k):
        pass

    def info(self):
        return _FakeInfo()

    def sync(self):
        pass

    def read_state(self, k, out=None):
        pass

    def obs(self, k):
        return {}


def _timed_paths_worker(rank, world, port, out_dir):
    import types

    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_1004_0023_gb300 import instances

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    _FakeEvent.rank = rank

    class _Pinned:  # from_numpy(...).pin_memory() without a GPU
        def __init__(self, t):
            self.t = t

        def pin_memory(self):
            return self.t

    fake_torch = types.SimpleNamespace(
        cuda=types.SimpleNamespace(Event=_FakeEvent, Stream=lambda: types.SimpleNamespace(cuda_stream=1),
                                   synchronize=lambda: None),
        from_numpy=lambda a: _Pinned(torch.from_numpy(a)),
        empty=lambda shape, dtype: _Pinned(torch.empty(shape, dtype=dtype)),
        int8=torch.int8)
    fake_pt = types.SimpleNamespace(PT=_FakeCtx, Batch=_FakeBatch)
    args = bench.parse_args(["--steps", "2", "--warmup", "3", "--batch-count", "6", "--batch-sweeps", "10",
                             "--no-cpu-baseline"])
    prob = instances.workload("regular3_n16_p32_r16", 1)
    e2e = bench.plain_e2e(args, prob, fake_pt, fake_torch, world, "cpu")
    b = bench.batched_headline(args, fake_pt, instances, fake_torch, 152, rank, world, rank, "cpu")
    mine = sum(p.attempts_per_sweep * p.n_sweeps
               for p in instances.batch_problems(count=6, index=1 + rank, n_sweeps=10))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "timed%d.json" % rank), "w") as f:
        json.dump({"e2e": e2e["value"], "e2e_ms": e2e["ms_per_step"], "value": b["value"],
                   "ms": b["ms_per_step"], "attempts": b["config"]["attempts_per_step"] * 2 / 2,
                   "plain_ms": b["plain_ms"], "frac": b["roofline"]["frac"], "batched_e2e": b["e2e"]["value"],
                   "units_e2e": b["e2e"]["value"] * b["e2e"]["ms_per_step"] / 1e3, "mine": float(mine)}, f)


def test_end_to_end_and_batched_figures_are_whole_job_over_ranks(tmp_path):
    """bench.plain_e2e and bench.batched_headline (with its plain comparison and e2e legs) on
    two gloo ranks with fake device objects (rank r's batched launch takes 10 (r + 1) ms): the
    values are the units of both ranks over the slowest rank's time, and the batched roofline
    stays per GPU."""
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_timed_paths_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / ("timed%d.json" % k))) for k in range(2)]
    total = r[0]["mine"] + r[1]["mine"]
    for k in range(2):
        assert r[k]["ms"] == 20.0 and r[k]["plain_ms"] == 20.0
        assert r[k]["value"] == pytest.approx(total / 0.020)
        assert r[k]["e2e"] == pytest.approx(r[0]["e2e"])  # one reduced figure, the same on every rank
        assert r[k]["batched_e2e"] == pytest.approx(r[0]["batched_e2e"])
        assert r[k]["units_e2e"] == pytest.approx(total)  # both ranks' attempts per e2e step
    # per-GPU roofline: rank k ran its own attempts in 10 (k + 1) ms, so its fraction of one
    # GPU's issue peak (152 SMs x 128 lanes x 2070 MHz) implies 31 to 40 instructions per attempt
    # (22 + 3d for degree 3 to 6; the whole-job rate would put rank 1 near twice that)
    peak = 152 * 128 * 2070e6
    for k in range(2):
        per_attempt = r[k]["frac"] * peak * (0.010 * (k + 1)) / r[k]["mine"]
        assert 31.0 <= per_attempt <= 40.0, (k, per_attempt)
