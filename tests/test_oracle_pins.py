"""Pins of the CPU oracle to things other than itself (all CPU-only).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign,
a wrong neighbour or slice index, a wrong update order, a swapped operand) fails it:

- Philox4x32-10 against curand's host generator (a library, run, not read);
- det_exp against libm exp (<= 2 ulp);
- deterministic tables: all-accept negates every spin, all-reject freezes the state;
- a hand-worked greedy sweep (tests/golden) fixes the site order and the even-then-odd
  copy order of Sec. 5;
- sampled moments against brute-force enumeration of exp(-S) and against the transfer
  matrix Z = Tr T^P, per rung, with swaps on;
- the ST energy estimator against exact diagonalisation and the N=1 closed form;
- swap acceptance against min(1, e^Delta) and the equal-rung special case;
- invariants (incremental E, M equal recomputed values; counters; permutation).
"""
import ctypes
import ctypes.util
import json
import os

import numpy as np
import pytest

import exact
from oracle import Oracle, det_exp, philox
from paper_1004_0023_gb300 import instances

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------- Philox

def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
                  "/usr/local/cuda/targets/x86_64-linux/lib", ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                continue
    return None


def _curand_host_philox(lib, seed, offset, count):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_uint64(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_uint64(offset)) == 0
        buf = np.zeros(count, np.uint32)
        assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
        return buf
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x5EED0001, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    """curand's host Philox4x32-10 emits block B = philox((B>>16 lo, B>>16 hi, B&0xffff, 0), seed)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    key = (seed & 0xFFFFFFFF, seed >> 32)
    blocks = [0, 1, 2, 7, 65535, 65536, 65537, 2 * 65536 + 3]
    for B in blocks:
        got = _curand_host_philox(lib, seed, 4 * B, 4)
        ref = philox((B >> 16 & 0xFFFFFFFF, B >> 48, B & 0xFFFF, 0), key)
        assert np.array_equal(got, ref), (hex(seed), B)
    # counter word 1 via a block index >= 2^48
    B = (1 << 48) * 3 + (5 << 16) + 9
    got = _curand_host_philox(lib, seed, 4 * B, 4)
    ref = philox(((B >> 16) & 0xFFFFFFFF, B >> 48, B & 0xFFFF, 0), key)
    assert np.array_equal(got, ref)


# ----------------------------------------------------------------------------- det_exp

def test_det_exp_within_two_ulp_of_libm():
    x = np.concatenate([np.linspace(-22.999, 0.0, 400001), -np.logspace(-300, 1.3, 2000),
                        np.array([0.0, -1e-300, -np.log(2), -22.18, -22.99999])])
    y = det_exp(x)
    ref = np.exp(x)
    ulp = np.abs(y - ref) / np.spacing(ref)
    assert ulp.max() <= 2.0, float(ulp.max())
    assert det_exp(np.array([0.0]))[0] == 1.0


# ----------------------------------------------------------------------------- tables

def _line_problem(P=4, R=1):
    # path 0-1-2, J01=+1 (antiferromagnetic), J12=-2, fields (1, 0, -1)
    return instances.tiny_problem(3, [(0, 1), (1, 2)], [1, -2], [1, 0, -1], P,
                                  [0.7] * R, [0.9] * R, seed=11)


def test_flip_table_matches_metropolis_probability():
    prob = instances.workload("regular3_n16_p32_r16", 1)
    o = Oracle.from_problem(prob)
    thr = o.flip_table().astype(np.float64)
    L = np.arange(-o.lmax, o.lmax + 1)[:, None]
    m = np.array([-2, 0, 2])[None, :]
    for r in range(prob.R):
        beta = 1.0 / prob.T[r]
        K = exact.coupling(beta, prob.gamma[r], prob.P)
        x = (2 * beta / prob.P) * L - 2 * K * m
        p = np.exp(np.minimum(x, 0.0))
        sentinel = thr[r] == 0xFFFFFFFF
        assert np.array_equal(sentinel, x >= -1e-12) or np.all(sentinel[x >= 0])
        fin = ~sentinel
        assert np.all(np.abs(thr[r][fin] - p[fin] * 2.0 ** 32) <= 1.0 + 1e-9 * p[fin] * 2.0 ** 32)


def test_all_accept_table_negates_every_spin():
    prob = instances.workload("regular3_n16_p32_r16", 2)
    probe = Oracle.from_problem(prob)
    nL = 2 * probe.lmax + 1
    thr = np.full((prob.R, nL, 3), 0xFFFFFFFF, np.uint32)
    o = Oracle.from_problem(prob, flip_thr=thr)
    x0 = o.read_state()
    ob0 = o.obs()
    o.sweep(1)
    x1 = o.read_state()
    assert np.array_equal(x1, -x0)
    ob = o.obs()
    assert np.all(ob["flip_acc"] == prob.n * prob.P)
    assert np.array_equal(ob["M"], ob0["M"])  # M is even in the spins
    _check_energies(prob, x1, ob)


def test_zero_table_freezes_state():
    prob = instances.workload("regular3_n16_p32_r16", 3)
    probe = Oracle.from_problem(prob)
    thr = np.zeros((prob.R, 2 * probe.lmax + 1, 3), np.uint32)
    o = Oracle.from_problem(prob, flip_thr=thr)
    x0 = o.read_state()
    o.sweep(5)
    assert np.array_equal(o.read_state(), x0)
    ob = o.obs()
    assert np.all(ob["flip_acc"] == 0) and np.all(ob["n_meas"] == 5)
    assert np.array_equal(ob["sum_E"], 5 * ob["E"])


def test_greedy_worked_example():
    """Hand-worked sweep (tests/golden/greedy_sweep_n3_p4.json) with 'flip iff L - m > 0'."""
    with open(os.path.join(HERE, "golden", "greedy_sweep_n3_p4.json")) as f:
        g = json.load(f)
    prob = instances.tiny_problem(g["n"], g["edges"], g["J"], g["h"], g["P"], [1.0], [1.0])
    lmax = g["lmax"]
    thr = np.zeros((1, 2 * lmax + 1, 3), np.uint32)
    for L in range(-lmax, lmax + 1):
        for mi, m in enumerate((-2, 0, 2)):
            if L - m > 0:
                thr[0, L + lmax, mi] = 0xFFFFFFFF
    o = Oracle.from_problem(prob, flip_thr=thr, swap_coef=np.zeros(0))
    assert o.lmax == lmax
    o.write_state(np.asarray(g["initial"], np.int8)[None])
    o.sweep(1)
    assert o.read_state()[0].tolist() == g["after_one_sweep"]
    assert int(o.obs()["flip_acc"][0]) == g["flips"]


# ----------------------------------------------------------------------------- sampling

def _check_energies(prob, x, ob):
    """Incremental E and M equal the values recomputed from the state (definitions)."""
    s = x.astype(np.int64)
    Ek = (s[:, prob.ei, :] * s[:, prob.ej, :] * prob.J[None, :, None]).sum(1) + (
        s * prob.h[None, :, None]).sum(1)
    assert np.array_equal(Ek.sum(1), ob["E"])
    M = (s * np.roll(s, -1, axis=2)).sum((1, 2))
    assert np.array_equal(M, ob["M"])


def _moments(o, n_batches, per_batch):
    """Batch means of E, M, E^2 per rung from the oracle's own int64 accumulators."""
    rows = []
    prev = o.obs()
    for _ in range(n_batches):
        o.run(per_batch, 1)
        cur = o.obs()
        dn = (cur["n_meas"] - prev["n_meas"]).astype(np.float64)
        rows.append(np.stack([(cur["sum_E"] - prev["sum_E"]) / dn, (cur["sum_M"] - prev["sum_M"]) / dn,
                              (cur["sum_E2"] - prev["sum_E2"]) / dn, (cur["sum_M2"] - prev["sum_M2"]) / dn]))
        prev = cur
    a = np.asarray(rows)
    return a.mean(0), a.std(0, ddof=1) / np.sqrt(n_batches)


def test_single_rung_matches_brute_force_enumeration():
    prob = _line_problem(P=4, R=1)
    ex = exact.enumerate_st(prob, 0)
    o = Oracle.from_problem(prob)
    mean, se = _moments(o, 40, 5000)
    for j, key in enumerate(("E", "M", "E2", "M2")):
        assert abs(mean[j, 0] - ex[key]) < 5 * se[j, 0] + 1e-9, (key, mean[j, 0], ex[key], se[j, 0])


def test_parallel_tempering_rung_marginals_match_enumeration():
    """Three rungs with swaps after every sweep: each rung samples its own exp(-S_r)."""
    prob = instances.tiny_problem(2, [(0, 1)], [2], [1, -1], 4, [0.5, 1.0, 2.0], [0.3, 0.8, 1.6],
                                  seed=5)
    o = Oracle.from_problem(prob)
    mean, se = _moments(o, 40, 5000)
    for r in range(prob.R):
        ex = exact.enumerate_st(prob, r)
        for j, key in enumerate(("E", "M", "E2", "M2")):
            assert abs(mean[j, r] - ex[key]) < 5 * se[j, r] + 1e-9, (r, key, mean[j, r], ex[key])
    ob = o.obs()
    assert np.all(ob["swap_acc"] > 0) and np.all(ob["swap_acc"] < ob["swap_att"])


def test_rung0_state_histogram_matches_enumeration():
    prob = instances.tiny_problem(2, [(0, 1)], [-1], [1, 0], 4, [0.8, 1.6], [0.5, 1.2], seed=9)
    ex = exact.enumerate_st(prob, 0)
    o = Oracle.from_problem(prob)
    counts = np.zeros(ex["prob"].size)
    n = 60000
    for _ in range(n):
        o.run(1, 1)
        counts[exact.state_code(o.read_state()[0])] += 1
    # G-test of the empirical histogram with a generous threshold for autocorrelation
    expected = ex["prob"] * n
    big = expected > 20
    tv = 0.5 * np.abs(counts / n - ex["prob"]).sum()
    assert tv < 0.03, tv
    rel = np.abs(counts[big] - expected[big]) / np.sqrt(expected[big])
    assert rel.max() < 8, rel.max()


def test_transfer_matrix_moments_at_larger_P():
    """N=6 prism graph, P=16, four rungs with swaps: <E>, <M> per rung vs Tr T^P."""
    edges = [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3), (0, 3), (1, 4), (2, 5)]
    prob = instances.tiny_problem(6, edges, [1, -2, 1, 2, -1, -1, 1, -2, 2], [1, 0, -1, 0, 1, 0], 16,
                                  [0.6, 0.8, 1.1, 1.5], [0.4, 0.8, 1.4, 2.2], seed=21)
    o = Oracle.from_problem(prob)
    mean, se = _moments(o, 40, 1500)
    for r in range(prob.R):
        ex = exact.transfer_matrix(prob, r)
        assert abs(mean[0, r] - ex["E"]) < 5 * se[0, r], (r, "E", mean[0, r], ex["E"], se[0, r])
        assert abs(mean[1, r] - ex["M"]) < 5 * se[1, r], (r, "M", mean[1, r], ex["M"], se[1, r])


def test_transfer_matrix_agrees_with_enumeration():
    prob = _line_problem(P=4, R=1)
    tm = exact.transfer_matrix(prob, 0)
    en = exact.enumerate_st(prob, 0)
    assert abs(tm["E"] - en["E"]) < 1e-9 and abs(tm["M"] - en["M"]) < 1e-9


def test_st_mapping_converges_to_exact_diagonalisation():
    """The estimator on exact ST moments approaches thermal <H> as P grows (error O(1/P^2))."""
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]
    prob = instances.tiny_problem(4, edges, [1, -1, 2, 1, -1], [1, 0, -1, 0], 8, [0.7], [1.3])
    ed = exact.exact_diag(prob, 0)
    est = {}
    for P in (32, 64, 128):
        tm = exact.transfer_matrix(prob, 0, P=P)
        est[P] = exact.st_energy_estimator(tm["E"], tm["M"], prob.n, P, 1 / prob.T[0], prob.gamma[0])
    err = {P: abs(est[P] - ed) for P in est}
    assert err[128] < err[64] < err[32]
    assert 3.0 < err[64] / err[128] < 5.0  # second-order Trotter error
    richardson = (4 * est[128] - est[64]) / 3
    assert abs(richardson - ed) < 1e-4 * max(1.0, abs(ed))


def test_single_spin_estimator_closed_form():
    """N=1, h=0: the ST estimator on the exact ST moments equals -Gamma tanh(beta Gamma) at
    every P (pins the coupling K and the estimator used by the checks below)."""
    for P, beta, g in ((4, 1.5, 0.8), (8, 0.7, 2.0), (16, 3.0, 0.4)):
        prob = instances.tiny_problem(1, [], [], [0], P, [1 / beta], [g])
        en = exact.enumerate_st(prob, 0)
        est = exact.st_energy_estimator(en["E"], en["M"], 1, P, beta, g)
        assert abs(est - (-g * np.tanh(beta * g))) < 1e-12


def test_single_spin_with_field_matches_enumeration():
    prob = instances.tiny_problem(1, [], [], [1], 8, [1 / 1.5], [0.8], seed=3)
    ex = exact.enumerate_st(prob, 0)
    o = Oracle.from_problem(prob)
    mean, se = _moments(o, 40, 5000)
    for j, key in enumerate(("E", "M", "E2", "M2")):
        assert abs(mean[j, 0] - ex[key]) < 5 * se[j, 0] + 1e-9, (key, mean[j, 0], ex[key])


def test_zero_field_single_spin_is_deterministic_on_the_antialigned_set():
    """Degenerate case of the method: one spin, h=0, P=4. When s^0=-s^2 and s^1=-s^3 every
    copy has m=0, so Delta S=0 and the Metropolis rule flips it with certainty; the even
    copies flip, then the odd ones, so each sweep negates the chain and it never leaves
    that set (the fixed even/odd scan is reducible here)."""
    prob = instances.tiny_problem(1, [], [], [0], 4, [1.0], [0.8], seed=3)
    o = Oracle.from_problem(prob)
    x = np.array([[[1, 1, -1, -1]]], np.int8)
    o.write_state(x)
    for t in range(1, 7):
        o.sweep(1)
        assert np.array_equal(o.read_state(), x * (-1) ** t)
    assert int(o.obs()["flip_acc"][0]) == 6 * 4


def test_oracle_energy_estimator_matches_exact_diagonalisation():
    edges = [(0, 1), (1, 2)]
    prob = instances.tiny_problem(3, edges, [1, -1], [1, 0, -1], 32, [1.0], [1.0], seed=13)
    ed = exact.exact_diag(prob, 0)
    tm = exact.transfer_matrix(prob, 0)
    trotter = abs(exact.st_energy_estimator(tm["E"], tm["M"], 3, 32, 1.0, 1.0) - ed)
    o = Oracle.from_problem(prob)
    rows = []
    prev = o.obs()
    for _ in range(40):
        o.run(2500, 1)
        cur = o.obs()
        dn = cur["n_meas"][0] - prev["n_meas"][0]
        rows.append(exact.st_energy_estimator((cur["sum_E"][0] - prev["sum_E"][0]) / dn,
                                              (cur["sum_M"][0] - prev["sum_M"][0]) / dn, 3, 32, 1.0, 1.0))
        prev = cur
    rows = np.asarray(rows)
    se = rows.std(ddof=1) / np.sqrt(rows.size)
    assert abs(rows.mean() - ed) < 5 * se + trotter, (rows.mean(), ed, se, trotter)


# ----------------------------------------------------------------------------- swaps

def test_equal_rungs_always_swap():
    prob = instances.tiny_problem(3, [(0, 1), (1, 2)], [1, 1], [0, 1, 0], 4, [0.5] * 4, [1.0] * 4)
    o = Oracle.from_problem(prob)
    assert np.all(o.swap_coef() == 0.0)
    for q in range(6):
        before = o.obs()["replica_at"].copy()
        o.swap()
        after = o.obs()["replica_at"]
        expect = before.copy()
        for r in range(q & 1, prob.R - 1, 2):
            expect[r], expect[r + 1] = before[r + 1], before[r]
        assert np.array_equal(after, expect)
    ob = o.obs()
    assert np.array_equal(ob["swap_acc"], ob["swap_att"]) and ob["swap_att"].sum() == 9


def test_swap_acceptance_frequency_is_metropolis():
    """Frozen chains on two rungs: from the unfavourable side swaps succeed with prob e^Delta."""
    prob = instances.tiny_problem(2, [(0, 1)], [1], [1, 0], 4, [1.0, 1.0], [0.6, 1.2], seed=77)
    probe = Oracle.from_problem(prob)
    thr = np.zeros((2, 2 * probe.lmax + 1, 3), np.uint32)
    o = Oracle.from_problem(prob, flip_thr=thr)
    x = np.ones((2, 2, 4), np.int8)
    x[1, 0, 1] = x[1, 1, 3] = -1
    o.write_state(x)
    a, c = o.swap_coef()
    ob = o.obs()
    E, M = ob["E"].astype(float), ob["M"].astype(float)
    delta = a * (E[0] - E[1]) + c * (M[0] - M[1])
    assert delta < 0
    tries = acc = 0
    for _ in range(60000):
        ob = o.obs()
        unfav = ob["replica_at"][0] == 0
        o.swap()  # even pass: pair (0,1)
        if unfav:
            tries += 1
            acc += int(o.obs()["replica_at"][0] == 1)
        o.swap()  # odd pass: no pair for R=2
    p = np.exp(delta)
    assert abs(acc / tries - p) < 5 * np.sqrt(p * (1 - p) / tries), (acc / tries, p)


# ----------------------------------------------------------------------------- invariants

@pytest.mark.parametrize("name", ["regular3_n16_p32_r16"])
def test_invariants_over_a_run(name):
    prob = instances.workload(name, 4)
    o = Oracle.from_problem(prob)
    for chunk in (1, 7, 50):
        o.run(chunk, 1)
        ob = o.obs()
        _check_energies(prob, o.read_state(), ob)
        assert sorted(ob["replica_at"].tolist()) == list(range(prob.R))
        assert np.all(ob["n_meas"] == ob["t"])
        assert np.all(ob["flip_acc"] <= prob.n * prob.P * ob["t"])
        assert np.all(ob["swap_acc"] <= ob["swap_att"])
        assert ob["swap_att"].sum() == sum(len(range(q & 1, prob.R - 1, 2)) for q in range(ob["q"]))


def test_run_equals_sweep_swap_loop_and_threads_are_bit_identical():
    prob = instances.workload("regular3_n16_p32_r16", 5)
    a = Oracle.from_problem(prob)
    b = Oracle.from_problem(prob, threads=4)
    a.run(60, 3)
    for _ in range(20):
        b.sweep(3)
        b.swap()
    assert np.array_equal(a.read_state(), b.read_state())
    oa, ob = a.obs(), b.obs()
    for k in oa:
        assert np.array_equal(np.asarray(oa[k]), np.asarray(ob[k])), k


def test_create_rejects_invalid_input():
    good = dict(n=3, ei=[0, 1], ej=[1, 2], J=[1, 1], h=[0, 0, 0], P=4, T=[1.0], gamma=[1.0], seed=1)
    Oracle(**good)
    for bad in (dict(P=3), dict(P=0), dict(J=[1, 0]), dict(ej=[0, 2]), dict(ej=[1, 3]),
                dict(ei=[0, 1, 1], ej=[1, 2, 0], J=[1, 1, 1]), dict(T=[0.0]), dict(gamma=[-1.0])):
        kw = dict(good, **bad)
        with pytest.raises(ValueError):
            Oracle(**kw)


# ----------------------------------------------------------------------------- classical PT
# P = 1 with Gamma = 0: classical parallel tempering over T (one copy per chain, no Trotter
# coupling). Pinned to the Boltzmann distribution exp(-beta E) enumerated over all 2^N states.

def _classical_problem(seed=31):
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (0, 3), (1, 4)]
    return instances.tiny_problem(6, edges, [1, -2, 1, -1, 2, -1, 1, -2], [1, 0, -1, 0, 1, 0], 1,
                                  [0.7, 1.4, 3.0], [0.0, 0.0, 0.0], seed=seed)


def test_classical_pt_samples_the_boltzmann_distribution_at_every_temperature():
    prob = _classical_problem()
    s, E = exact.slice_energies(prob.n, prob.ei, prob.ej, prob.J, prob.h)
    o = Oracle.from_problem(prob)
    o.run(2000, 1)
    rows, rows2 = [], []
    prev = o.obs()
    for _ in range(40):
        o.run(2000, 1)
        cur = o.obs()
        dn = np.asarray(cur["n_meas"]) - np.asarray(prev["n_meas"])
        rows.append((np.asarray(cur["sum_E"]) - np.asarray(prev["sum_E"])) / dn)
        rows2.append((np.asarray(cur["sum_E2"]) - np.asarray(prev["sum_E2"])) / dn)
        assert np.all(np.asarray(cur["M"]) == prob.n)  # one copy: M = sum_i s_i s_i
        prev = cur
    rows, rows2 = np.asarray(rows), np.asarray(rows2)
    for r in range(prob.R):
        w = np.exp(-(E - E.min()) / prob.T[r])
        w /= w.sum()
        for got, want in ((rows[:, r], float(w @ E)), (rows2[:, r], float(w @ E ** 2))):
            se = got.std(ddof=1) / np.sqrt(got.size)
            assert abs(got.mean() - want) < 5 * se + 1e-12, (r, got.mean(), want, se)
    assert np.all(np.asarray(prev["swap_acc"]) > 0)


def test_classical_table_ignores_the_trotter_column_and_swaps_see_only_energy():
    prob = _classical_problem()
    o = Oracle.from_problem(prob)
    thr = o.flip_table().reshape(prob.R, -1, 3)
    assert np.all(thr[:, :, 0] == thr[:, :, 1]) and np.all(thr[:, :, 1] == thr[:, :, 2])
    coef = o.swap_coef()
    assert np.all(coef[prob.R - 1:] == 0.0) and np.all(coef[: prob.R - 1] > 0.0)
    # L >= 0 always flips; the least favourable move is the rarest at the coldest rung
    lmax = (thr.shape[1] - 1) // 2
    assert np.all(thr[:, lmax:, :] == 0xFFFFFFFF)
    assert thr[0, 0, 0] < thr[-1, 0, 0]


def test_classical_mode_needs_gamma_zero_and_quantum_mode_needs_gamma_positive():
    prob = _classical_problem()
    bad = instances.tiny_problem(6, list(zip(prob.ei, prob.ej)), prob.J, prob.h, 1, prob.T, [0.0, 0.5, 0.0])
    with pytest.raises(Exception):
        Oracle.from_problem(bad)
    quantum_zero = instances.tiny_problem(6, list(zip(prob.ei, prob.ej)), prob.J, prob.h, 2, prob.T, [0.0] * 3)
    with pytest.raises(Exception):
        Oracle.from_problem(quantum_zero)
