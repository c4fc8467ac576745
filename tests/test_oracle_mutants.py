"""Planted mistakes in the oracle are caught by its pins (CPU only).

Each mutant is a one-line textual change to a private copy of oracle/pt_oracle.c,
compiled into a temporary library. A compact battery of the pins from
test_oracle_pins.py runs against it and at least one check must fail. This shows the
pins constrain each part of the oracle (field, Trotter term, update order, table,
swap rule, statistics, Philox, det_exp) rather than only agreeing with it.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import exact
from oracle import oracle as orc
from paper_1004_0023_gb300 import instances

MUTANTS = {
    "drop_field_h": ("int32_t field = o->h[i];", "int32_t field = 0;"),
    "trotter_uses_k_minus_1_twice": ("*spin_ptr(o, rep, i, (k + 1) % P));", "*spin_ptr(o, rep, i, (k + P - 1) % P));"),
    "odd_copies_first": ("int32_t k = p + 2 * hh;", "int32_t k = (1 - p) + 2 * hh;"),
    "sites_in_reverse": ("int32_t si = *spin_ptr(o, rep, i, k);", "i = o->N - 1 - i; int32_t si = *spin_ptr(o, rep, i, k); i = o->N - 1 - i;"),
    "table_sign_of_m": ("double x = c1 * (double)L - c2 * (double)m;", "double x = c1 * (double)L + c2 * (double)m;"),
    "coupling_K_factor": (": -0.5 * log(tanh(a));", ": -1.0 * log(tanh(a));"),
    "energy_update_uses_m": ("dE -= 2 * (int64_t)L;", "dE -= 2 * (int64_t)m;"),
    "swap_delta_sign": ("double delta = a[r] * dE + c[r] * dM;", "double delta = a[r] * dE - c[r] * dM;"),
    "swap_coef_transposed": ("o->coef[r] = b[r] - b[r + 1];", "o->coef[r] = b[r + 1] - b[r];"),
    "swap_pair_parity": ("for (int32_t r = (int32_t)(o->q & 1); r + 1 < o->R; r += 2) {",
                         "for (int32_t r = (int32_t)((o->q + 1) & 1); r + 1 < o->R; r += 2) {"),
    "stat_E2_uses_M": ("o->sum_E2[r] += o->E[rep] * o->E[rep];", "o->sum_E2[r] += o->E[rep] * o->M[rep];"),
    "philox_c1_c3_swapped": ("uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;", "uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c3 ^ k0;"),
    "philox_key_bump": ("k1 += PHILOX_W1;", "k1 += PHILOX_W0;"),
    "det_exp_short_series": ("double p = inv_fact[13];\n    for (int k = 12;", "double p = inv_fact[9];\n    for (int k = 8;"),
    "flip_word_shared": ("u[hh & 3] < th", "u[0] < th"),
    "classical_keeps_trotter_term": ("int32_t m = P == 1 ? 0", "int32_t m = P == 0 ? 0"),
    "classical_keeps_coupling": ("K[r] = o->P == 1 ? 0.0 :", "K[r] = o->P == 0 ? 0.0 :"),
}


def _battery(lib):
    """Returns the names of failed checks (empty = mutant survives)."""
    failed = []

    def check(name, fn):
        try:
            if not fn():
                failed.append(name)
        except Exception:  # a crash also counts as detection
            failed.append(name)

    # greedy worked example
    import json
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "golden", "greedy_sweep_n3_p4.json")) as f:
        g = json.load(f)

    def greedy():
        prob = instances.tiny_problem(g["n"], g["edges"], g["J"], g["h"], g["P"], [1.0], [1.0])
        lm = g["lmax"]
        thr = np.zeros((1, 2 * lm + 1, 3), np.uint32)
        for L in range(-lm, lm + 1):
            for mi, m in enumerate((-2, 0, 2)):
                if L - m > 0:
                    thr[0, L + lm, mi] = 0xFFFFFFFF
        o = orc.Oracle.from_problem(prob, flip_thr=thr, swap_coef=np.zeros(0), lib=lib)
        o.write_state(np.asarray(g["initial"], np.int8)[None])
        o.sweep(1)
        return o.read_state()[0].tolist() == g["after_one_sweep"]

    def invariants():
        prob = instances.workload("regular3_n16_p32_r16", 4)
        o = orc.Oracle.from_problem(prob, lib=lib)
        o.run(20, 1)
        ob = o.obs()
        s = o.read_state().astype(np.int64)
        Ek = (s[:, prob.ei, :] * s[:, prob.ej, :] * prob.J[None, :, None]).sum(1) + (
            s * prob.h[None, :, None]).sum(1)
        M = (s * np.roll(s, -1, axis=2)).sum((1, 2))
        return np.array_equal(Ek.sum(1), ob["E"]) and np.array_equal(M, ob["M"])

    def moments():
        prob = instances.tiny_problem(2, [(0, 1)], [2], [1, -1], 4, [0.5, 1.0, 2.0], [0.3, 0.8, 1.6], seed=5)
        o = orc.Oracle.from_problem(prob, lib=lib)
        rows, prev = [], o.obs()
        for _ in range(20):
            o.run(4000, 1)
            cur = o.obs()
            dn = (cur["n_meas"] - prev["n_meas"]).astype(float)
            rows.append(np.stack([(cur[k] - prev[k]) / dn for k in ("sum_E", "sum_M", "sum_E2")]))
            prev = cur
        a = np.asarray(rows)
        mean, se = a.mean(0), a.std(0, ddof=1) / np.sqrt(a.shape[0])
        for r in range(prob.R):
            ex = exact.enumerate_st(prob, r)
            for j, key in enumerate(("E", "M", "E2")):
                if abs(mean[j, r] - ex[key]) > 5 * se[j, r] + 1e-9:
                    return False
        return True

    def equal_rungs():
        prob = instances.tiny_problem(3, [(0, 1), (1, 2)], [1, 1], [0, 1, 0], 4, [0.5] * 4, [1.0] * 4)
        o = orc.Oracle.from_problem(prob, lib=lib)
        o.swap()
        return o.obs()["replica_at"].tolist() == [1, 0, 3, 2]

    def swap_frequency():
        prob = instances.tiny_problem(2, [(0, 1)], [1], [1, 0], 4, [1.0, 1.0], [0.6, 1.2], seed=77)
        thr = np.zeros((2, 2 * 2 + 1, 3), np.uint32)
        o = orc.Oracle.from_problem(prob, flip_thr=thr, lib=lib)
        x = np.ones((2, 2, 4), np.int8)
        x[1, 0, 1] = x[1, 1, 3] = -1
        o.write_state(x)
        K = [exact.coupling(1.0, g, 4) for g in prob.gamma]
        ob = o.obs()
        delta = (K[1] - K[0]) * float(ob["M"][0] - ob["M"][1])  # equal T: only the Trotter term
        tries = acc = 0
        for _ in range(20000):
            unfav = o.obs()["replica_at"][0] == 0
            o.swap()
            if unfav:
                tries += 1
                acc += int(o.obs()["replica_at"][0] == 1)
            o.swap()
        p = np.exp(min(delta, 0.0))
        return abs(acc / tries - p) < 5 * np.sqrt(p * (1 - p) / tries) + 1e-12

    def philox_curand():
        import test_oracle_pins as pins
        cur = pins._curand()
        if cur is None:
            return True
        seed = 0x123456789ABCDEF
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for B in (0, 65537, (1 << 48) * 3 + (5 << 16) + 9):
            got = pins._curand_host_philox(cur, seed, 4 * B, 4)
            if not np.array_equal(got, orc.philox(((B >> 16) & 0xFFFFFFFF, B >> 48, B & 0xFFFF, 0), key, lib=lib)):
                return False
        return True

    def det_exp_ulp():
        x = np.linspace(-22.999, 0.0, 20001)
        y = orc.det_exp(x, lib=lib)
        return (np.abs(y - np.exp(x)) / np.spacing(np.exp(x))).max() <= 2.0

    def classical():
        edges = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]
        prob = instances.tiny_problem(4, edges, [1, -2, 1, 2, -1], [1, 0, -1, 0], 1, [0.8, 2.0], [0.0, 0.0], seed=9)
        o = orc.Oracle.from_problem(prob, lib=lib)
        s, E = exact.slice_energies(prob.n, prob.ei, prob.ej, prob.J, prob.h)
        rows, prev = [], o.obs()
        for _ in range(20):
            o.run(3000, 1)
            cur = o.obs()
            if not np.all(np.asarray(cur["M"]) == prob.n):
                return False
            rows.append((cur["sum_E"] - prev["sum_E"]) / (cur["n_meas"] - prev["n_meas"]).astype(float))
            prev = cur
        a = np.asarray(rows)
        mean, se = a.mean(0), a.std(0, ddof=1) / np.sqrt(a.shape[0])
        for r in range(prob.R):
            w = np.exp(-(E - E.min()) / prob.T[r])
            if abs(mean[r] - float(w @ E) / w.sum()) > 5 * se[r] + 1e-9:
                return False
        return True

    for name, fn in (("greedy", greedy), ("invariants", invariants), ("moments", moments), ("classical", classical),
                     ("equal_rungs", equal_rungs), ("swap_frequency", swap_frequency),
                     ("philox", philox_curand), ("det_exp", det_exp_ulp)):
        check(name, fn)
    return failed


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="orc_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


def test_unmutated_oracle_passes_battery(workdir):
    assert _battery(orc.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, workdir):
    src = open(orc.SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, "mutation site not found: " + name
    mdir = os.path.join(workdir, name)
    os.makedirs(mdir)
    shutil.copy(orc.HDR, mdir)
    msrc = os.path.join(mdir, "pt_oracle.c")
    with open(msrc, "w") as f:
        f.write(src.replace(old, new))
    out = os.path.join(mdir, "liboracle_mut.so")
    subprocess.run(["gcc", *orc.CFLAGS, "-I", mdir, "-o", out, msrc, "-lm"], check=True)
    failed = _battery(orc.load(out))
    assert failed, "mutant %s survived every pin" % name
