"""pt_run_noalloc against pt_run and the CPU oracle: same bits on two calls in a row.

pt_run_noalloc serves callers that cannot allocate device memory (allocator-free latency
loops, runtimes and frameworks that hand out device memory only from their own pool). Here
the test itself owns the device buffers (torch tensors) and fills them from the host-only
helpers; the entry point must leave exactly the state pt_run leaves on a context, and the
state the oracle reaches. The tolerance is the one every parity test here uses: zero.
The cases cover one launch per call, calls that need several launches (more swap passes x
rungs than the fixed mailbox array holds, so the mailboxes are cleared between launches on
one stream), and calls whose sweep count is not a multiple of the swap interval.
"""
import ctypes

import numpy as np
import pytest

from paper_1004_0023_gb300 import instances
from paper_1004_0023_gb300 import pt

pytestmark = pytest.mark.gpu


def _device_problem(torch, prob, ref, stream):
    """Caller-owned device buffers for prob, in the layout include/pt.h documents."""
    n, P, R = prob.n, prob.P, prob.R
    adj = [[] for _ in range(n)]
    for a, b, J in zip(prob.ei, prob.ej, prob.J):
        adj[a].append((b, J))
        adj[b].append((a, J))
    deg = max(len(x) for x in adj)
    stride = 4 if deg <= 4 else (8 if deg <= 8 else 32)
    nbr = np.zeros((n, stride), np.uint32)
    for i in range(n):
        for d in range(stride):
            j, J = adj[i][d] if d < len(adj[i]) else (i, 0)
            nbr[i, d] = (j << 8) | (int(J) & 0xFF)
    items, off = pt.make_schedule(n, prob.ei, prob.ej)
    lmax = ref.info.lmax
    thr, coef = pt.make_tables(P, prob.T, prob.gamma, lmax)
    coef = coef if coef.size else np.zeros(2, np.float64)
    slot_stride = (n * P + 15) // 16 * 16
    x0 = ref.read_state()  # identity permutation before the first swap: rung order == replica order
    spins = np.zeros((R, slot_stride), np.int8)
    spins[:, : n * P] = x0.reshape(R, n * P)
    ob = ref.obs()
    assert np.array_equal(ob["replica_at"], np.arange(R))
    dev = torch.device("cuda")
    t = {
        "nbr": torch.from_numpy(nbr.view(np.int32)).to(dev),
        "h": torch.from_numpy(prob.h.astype(np.int8)).to(dev),
        "items": torch.from_numpy(items.view(np.int32)).to(dev),
        "level_off": torch.from_numpy(off.astype(np.int32)).to(dev),
        "thr": torch.from_numpy(thr.reshape(-1).view(np.int32)).to(dev),
        "coef": torch.from_numpy(coef).to(dev),
        "spins": torch.from_numpy(spins).to(dev),
        "E": torch.from_numpy(ob["E"].copy()).to(dev),
        "M": torch.from_numpy(ob["M"].copy()).to(dev),
        "rung_of_slot": torch.arange(R, dtype=torch.int32, device=dev),
        "slot_of_rung": torch.arange(R, dtype=torch.int32, device=dev),
        "stats": torch.zeros(R * 6, dtype=torch.int64, device=dev),
        "swap_stats": torch.zeros(R * 2, dtype=torch.int64, device=dev),
        "status": torch.zeros(4, dtype=torch.int32, device=dev),
    }
    torch.cuda.synchronize()
    dp = pt.pt_device_problem(n, P, R, lmax, stride, int(off.size - 1),
                              *[ctypes.c_void_p(t[k].data_ptr()) for k in
                                ("nbr", "h", "items", "level_off", "thr", "coef", "spins", "E", "M",
                                 "rung_of_slot", "slot_of_rung", "stats", "swap_stats", "status")],
                              prob.seed & 0xFFFFFFFFFFFFFFFF, 0, 0)
    return dp, t


def _state_of(torch, t, prob):
    """Rung-ordered spins and per-rung statistics from the caller-owned buffers."""
    torch.cuda.synchronize()
    n, P, R = prob.n, prob.P, prob.R
    slot_of = t["slot_of_rung"].cpu().numpy()
    spins = t["spins"].cpu().numpy()[:, : n * P].reshape(R, n, P)
    stats = t["stats"].cpu().numpy().reshape(R, 6)
    sw = t["swap_stats"].cpu().numpy().reshape(R, 2)
    E, M = t["E"].cpu().numpy(), t["M"].cpu().numpy()
    return {
        "state": spins[slot_of], "E": E[slot_of], "M": M[slot_of], "n_meas": stats[:, 0], "sum_E": stats[:, 1],
        "sum_E2": stats[:, 2], "sum_M": stats[:, 3], "sum_M2": stats[:, 4], "flip_acc": stats[:, 5],
        "swap_att": sw[: R - 1, 0], "swap_acc": sw[: R - 1, 1], "replica_at": slot_of,
        "status": int(t["status"].cpu().numpy()[0]),
    }


_KEYS = ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc", "swap_att", "swap_acc",
         "replica_at")


def _run_and_compare(torch, name, calls, sps, with_oracle=False):
    prob = instances.workload(name, 6)
    ref = pt.PT.from_problem(prob)
    orc = None
    if with_oracle:
        from oracle import Oracle

        orc = Oracle.from_problem(prob, threads=4)
    dp, bufs = _device_problem(torch, prob, ref, None)
    stream = torch.cuda.Stream()
    for n_sweeps in calls:
        pt.run_noalloc(dp, n_sweeps, sps, 0, stream.cuda_stream)
        dp.t0 += n_sweeps
        dp.q0 += n_sweeps // sps
        ref.run(n_sweeps, sps)
        stream.synchronize()
        got = _state_of(torch, bufs, prob)
        assert got["status"] == 0
        wants = [("pt_run", ref.read_state(), ref.obs())]
        if orc is not None:
            orc.run(n_sweeps, sps)
            wants.append(("oracle", orc.read_state(), orc.obs()))
        for who, state, want in wants:
            assert np.array_equal(got["state"], state), (name, n_sweeps, who)
            for k in _KEYS:
                assert np.array_equal(np.asarray(got[k]), np.asarray(want[k])), (name, n_sweeps, who, k)
        assert int(ref.obs()["t"]) == dp.t0 and int(ref.obs()["q"]) == dp.q0
    ref.close()
    if orc is not None:
        orc.close()


@pytest.mark.parametrize("name,calls", [("regular3_n16_p32_r16", (300, 211)), ("regular3_n256_p64_r64", (120, 80))])
def test_noalloc_entry_point_matches_pt_run_on_two_calls_in_a_row(libpt, name, calls):
    torch = pytest.importorskip("torch")
    _run_and_compare(torch, name, calls, 1)


def test_noalloc_entry_point_matches_the_oracle_on_two_calls_in_a_row(libpt):
    torch = pytest.importorskip("torch")
    _run_and_compare(torch, "regular3_n16_p32_r16", (257, 190), 1, with_oracle=True)


def test_noalloc_calls_that_need_several_launches(libpt):
    # R = 64 rungs leave room for 16384 / 64 = 256 swap passes per launch: 600 sweeps with a
    # swap after each run as three launches (256, 256, 88 passes), 300 as two, each clearing
    # the shared mailboxes it uses after the previous launch on the same stream
    torch = pytest.importorskip("torch")
    assert 600 * 64 > pt.PT_NOALLOC_MAILBOXES and 300 * 64 > pt.PT_NOALLOC_MAILBOXES
    _run_and_compare(torch, "regular3_n256_p64_r64", (600, 300), 1)


def test_noalloc_sweep_counts_that_are_not_a_multiple_of_the_swap_interval(libpt):
    # 301 = 100 intervals of 3 sweeps + 1 sweep without a pass; the second call starts on an
    # interval boundary of its own, as pt_run does; the second case also spans two launches
    torch = pytest.importorskip("torch")
    _run_and_compare(torch, "regular3_n16_p32_r16", (301, 152), 3, with_oracle=True)
    _run_and_compare(torch, "regular3_n256_p64_r64", (1003, 257), 2)


def test_noalloc_entry_point_rejects_sizes_beyond_its_fixed_scratch(libpt):
    # the size checks run before any device access, so placeholder addresses are never used
    dp = pt.pt_device_problem()
    dp.n, dp.P, dp.R, dp.lmax, dp.row_stride, dp.n_levels = 4, 4, 16385, 3, 4, 2
    for f in ("nbr", "h", "items", "level_off", "thr", "coef", "E", "M", "rung_of_slot", "slot_of_rung", "stats",
              "swap_stats", "status"):
        setattr(dp, f, 16)
    dp.spins = 256
    with pytest.raises(pt.PTError) as e:
        pt.run_noalloc(dp, 10, 1)
    assert e.value.code == pt.PT_EINVAL and "mailbox" in str(e.value)
