"""pt_run_noalloc against pt_run: same bits on two calls in a row.

pt_run_noalloc serves callers that cannot allocate device memory (stream capture into a
CUDA graph, allocator-free latency loops, runtimes with their own memory pool). Here the
test itself owns the device buffers (torch tensors) and fills them from the host-only
helpers; the entry point must leave exactly the state pt_run leaves on a context. The
tolerance is the one every parity test here uses: zero.
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


@pytest.mark.parametrize("name,calls", [("regular3_n16_p32_r16", (300, 211)), ("regular3_n256_p64_r64", (120, 80))])
def test_noalloc_entry_point_matches_pt_run_on_two_calls_in_a_row(libpt, name, calls):
    torch = pytest.importorskip("torch")
    prob = instances.workload(name, 6)
    ref = pt.PT.from_problem(prob)
    dp, bufs = _device_problem(torch, prob, ref, None)
    stream = torch.cuda.Stream()
    for n_sweeps in calls:
        pt.run_noalloc(dp, n_sweeps, 1, 0, stream.cuda_stream)
        dp.t0 += n_sweeps
        dp.q0 += n_sweeps
        ref.run(n_sweeps, 1)
        stream.synchronize()
        got = _state_of(torch, bufs, prob)
        want = ref.obs()
        assert got["status"] == 0
        assert np.array_equal(got["state"], ref.read_state())
        for k in ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc", "swap_att",
                  "swap_acc", "replica_at"):
            assert np.array_equal(np.asarray(got[k]), np.asarray(want[k])), (name, n_sweeps, k)
    ref.close()


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
