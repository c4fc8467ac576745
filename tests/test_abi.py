"""The C-ABI library builds, loads and exports every entry point of include/pt.h; its
host-only setup (FP64 tables, level schedule) matches the oracle and the sequential
order. No compute call needs a GPU here."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

from oracle import Oracle
from paper_1004_0023_gb300 import instances
from paper_1004_0023_gb300 import pt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pt_\w+)\s*\(", src, flags=re.M))
    return names


def test_every_declared_symbol_is_exported(libpt):
    names = declared_entry_points()
    assert {"pt_create", "pt_sweep", "pt_swap", "pt_run", "pt_read_state",
            "pt_read_observables"} <= names
    for n in sorted(names):
        assert hasattr(libpt, n), n
    assert names <= set(pt.exported_symbols()) | names


def test_create_without_device_fails_loudly(libpt):
    import conftest

    if conftest.has_gpu():
        pytest.skip("a GPU is present")
    prob = instances.workload("regular3_n16_p32_r16", 1)
    with pytest.raises(pt.PTError) as e:
        pt.PT.from_problem(prob)
    assert e.value.code in (pt.PT_ENODEV, pt.PT_ECUDA)


def test_create_rejects_out_of_range_instances_before_any_device_call(libpt):
    """pt_create checks its arguments on the host first, so each bad instance gets PT_EINVAL
    with or without a GPU: fields outside [-127, 127] (INT_MIN included, which must not reach
    abs()), |h| + sum |J| above 127, zero or out-of-range couplings, odd P, and a non-finite
    or non-positive rung."""
    prob = instances.workload("regular3_n16_p32_r16", 1)

    def create(h=None, J=None, P=None, T=None, gamma=None):
        return pt.PT(prob.n, prob.ei, prob.ej, prob.J if J is None else J, prob.h if h is None else h,
                     prob.P if P is None else P, prob.T if T is None else T,
                     prob.gamma if gamma is None else gamma, 1)

    bad = []
    for v in (-(2 ** 31), 128, -128, 2 ** 31 - 1):
        h = np.array(prob.h, np.int32)
        h[3] = v
        bad.append(dict(h=h))
    h = np.array(prob.h, np.int32)
    h[prob.ei[0]] = 127  # in range alone, but the site's couplings push the sum past 127
    bad.append(dict(h=h))
    for v in (0, 128, -(2 ** 31)):
        J = np.array(prob.J, np.int32)
        J[0] = v
        bad.append(dict(J=J))
    bad.append(dict(P=3))
    T = np.array(prob.T, np.float64)
    T[1] = np.inf
    bad.append(dict(T=T))
    g = np.array(prob.gamma, np.float64)
    g[2] = -1.0
    bad.append(dict(gamma=g))
    for kw in bad:
        with pytest.raises(pt.PTError) as e:
            create(**kw)
        assert e.value.code == pt.PT_EINVAL, kw


@pytest.mark.parametrize("name", ["regular3_n16_p32_r16", "regular3_n256_p64_r64", "chimera16_n2048_p128_r96",
                                  "classical_regular3_n256_r64"])
def test_host_tables_bit_identical_to_oracle(libpt, name):
    prob = instances.workload(name, 1)
    o = Oracle.from_problem(prob)
    thr, coef = pt.make_tables(prob.P, prob.T, prob.gamma, o.lmax)
    assert np.array_equal(thr, o.flip_table())
    assert np.array_equal(coef.view(np.uint64), o.swap_coef().view(np.uint64))


def test_host_tables_bit_identical_to_oracle_on_random_ladders(libpt):
    """The FP64 tables pt_create builds equal the oracle's bit for bit on random ladders:
    T and Gamma spread over four decades (so thresholds run from "always" through the
    exponential range down to 0), P from 1 (classical, Gamma = 0) to 4096, Lmax up to 127.
    A one-site instance with h = Lmax gives the oracle the same table size."""
    rng = np.random.default_rng(11)
    for _ in range(40):
        P = int(rng.choice([1, 2, 4, 8, 16, 32, 64, 128, 512, 4096]))
        R = int(rng.integers(1, 12))
        lmax = int(rng.integers(1, 128))
        T = 10.0 ** rng.uniform(-2.0, 2.0, R)
        gamma = np.zeros(R) if P == 1 else 10.0 ** rng.uniform(-2.0, 2.0, R)
        prob = instances.tiny_problem(1, [], [], [lmax], P, T, gamma)
        o = Oracle.from_problem(prob)
        assert o.lmax == lmax
        thr, coef = pt.make_tables(P, T, gamma, lmax)
        assert np.array_equal(thr, o.flip_table()), (P, R, lmax)
        assert np.array_equal(coef.view(np.uint64), o.swap_coef().view(np.uint64)), (P, R, lmax)
        o.close()


def test_host_tables_reject_bad_ladder(libpt):
    with pytest.raises(pt.PTError):
        pt.make_tables(4, [1.0, 0.0], [1.0, 1.0], 3)
    with pytest.raises(pt.PTError):
        pt.make_tables(3, [1.0], [1.0], 3)
    with pytest.raises(pt.PTError):  # classical chains (P = 1) need gamma = 0
        pt.make_tables(1, [1.0, 2.0], [0.0, 0.5], 3)
    with pytest.raises(pt.PTError):  # Trotter chains need gamma > 0
        pt.make_tables(2, [1.0, 2.0], [0.0, 0.0], 3)


def _check_schedule(n, ei, ej):
    items, off = pt.make_schedule(n, ei, ej)
    assert sorted(items.tolist()) == list(range(2 * n))
    level = np.empty(2 * n, np.int64)
    for l in range(off.size - 1):
        for it in items[off[l]:off[l + 1]]:
            level[it] = l
    adj = [set() for _ in range(n)]
    for a, b in zip(ei, ej):
        adj[a].add(b)
        adj[b].add(a)
    # every pair of conflicting updates keeps its sequential order (strictly earlier level)
    for i in range(n):
        assert level[2 * i] < level[2 * i + 1]
        for j in adj[i]:
            if j < i:
                assert level[2 * j] < level[2 * i]
                assert level[2 * j + 1] < level[2 * i + 1]
    # and the schedule is as short as the dependencies allow: each update at level l > 0
    # has a predecessor at level l - 1
    for i in range(n):
        for p in (0, 1):
            l = level[2 * i + p]
            if l == 0:
                continue
            preds = [level[2 * j + p] for j in adj[i] if j < i] + ([level[2 * i]] if p == 1 else [])
            assert max(preds) == l - 1
    return off.size - 1


def _levels(items, off):
    level = np.empty(items.size, np.int64)
    for l in range(off.size - 1):
        level[items[off[l]:off[l + 1]]] = l
    return level


def _rounds(off, per_round):
    return int(sum(-(-int(c) // per_round) for c in np.diff(off)))


@pytest.mark.parametrize("name,per_round,expect", [("regular3_n256_p64_r64", 48, 12),
                                                   ("chimera16_n2048_p128_r96", 32, 128),
                                                   ("regular3_n16_p32_r16", 96, 6)])
def test_balanced_schedule_keeps_dependencies_and_level_count(name, per_round, expect):
    """Rebalanced levels: a permutation of the updates, every dependency strictly earlier,
    the same level count as the as-early-as-possible schedule, and fewer kernel rounds
    (N=256: 16 -> 12 rounds of 48; the K4,4 lattice: 144 -> 128 rounds of 32, the bound
    4096 / 32)."""
    prob = instances.workload(name, 1)
    n = prob.n
    items0, off0 = pt.make_schedule(n, prob.ei, prob.ej)
    items, off = pt.make_schedule(n, prob.ei, prob.ej, items_per_round=per_round)
    assert sorted(items.tolist()) == list(range(2 * n))
    assert off.size == off0.size
    level = _levels(items, off)
    adj = [set() for _ in range(n)]
    for a, b in zip(prob.ei, prob.ej):
        adj[a].add(b)
        adj[b].add(a)
    for i in range(n):
        assert level[2 * i] < level[2 * i + 1]
        for j in adj[i]:
            if j < i:
                assert level[2 * j] < level[2 * i]
                assert level[2 * j + 1] < level[2 * i + 1]
    assert _rounds(off, per_round) <= _rounds(off0, per_round)
    assert _rounds(off, per_round) == expect


def test_balanced_schedule_degenerate_graphs():
    # no edges: two levels whatever the round size; a path: fully sequential, nothing to move
    for per_round in (1, 3, 100):
        items, off = pt.make_schedule(5, [], [], items_per_round=per_round)
        assert off.size == 3 and sorted(items.tolist()) == list(range(10))
        n = 6
        items, off = pt.make_schedule(n, list(range(n - 1)), list(range(1, n)), items_per_round=per_round)
        assert off.size - 1 == n + 1
        level = _levels(items, off)
        assert all(level[2 * i] == i and level[2 * i + 1] == i + 1 for i in range(n))
    with pytest.raises(pt.PTError):
        pt.make_schedule(4, [0], [1], items_per_round=-1)


def test_schedule_respects_sequential_order():
    for name in ("regular3_n16_p32_r16", "regular3_n256_p64_r64", "chimera16_n2048_p128_r96"):
        prob = instances.workload(name, 1)
        nlev = _check_schedule(prob.n, prob.ei, prob.ej)
        assert nlev < 2 * prob.n
    # a path 0-1-2-...: fully sequential even part, odd part one level behind
    n = 6
    nlev = _check_schedule(n, list(range(n - 1)), list(range(1, n)))
    assert nlev == n + 1
    # no edges: everything in two levels
    assert _check_schedule(5, [], []) == 2


def test_ctypes_structs_match_the_c_header(tmp_path):
    """Sizes and field offsets of every ABI struct agree between include/pt.h and pt.py."""
    import shutil
    import subprocess

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = {"pt_instance": pt.pt_instance, "pt_rung": pt.pt_rung, "pt_options": pt.pt_options,
               "pt_observables": pt.pt_observables, "pt_info": pt.pt_info, "pt_request": pt.pt_request,
               "pt_batch_info": pt.pt_batch_info, "pt_device_problem": pt.pt_device_problem,
               "pt_server_options": pt.pt_server_options, "pt_server_info": pt.pt_server_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pt.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines.append('printf("PT_NOALLOC_MAILBOXES %d\\n", PT_NOALLOC_MAILBOXES);')
    lines.append("return 0; }")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(out["PT_NOALLOC_MAILBOXES"]) == pt.PT_NOALLOC_MAILBOXES
    for name, cls in structs.items():
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(out["%s.%s" % (name, f[0])]) == getattr(cls, f[0]).offset, (name, f[0])


def _random_graph(kind, n, rng):
    if kind == "sparse":
        p = rng.uniform(0.0, min(1.0, 8.0 / n))
        return [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    if kind == "tree":
        return [(int(rng.integers(0, i)), i) for i in range(1, n)]
    if kind == "star":
        return [(0, i) for i in range(1, n)]
    if kind == "path":  # a path through the sites in random order: long dependency chains
        perm = rng.permutation(n)
        return [(int(perm[i]), int(perm[i + 1])) for i in range(n - 1)]
    ei, ej = instances.random_regular_graph(n, 3, rng)
    return list(zip(ei.tolist(), ej.tolist()))


@pytest.mark.parametrize("kind", ["sparse", "tree", "star", "path", "regular3"])
def test_balanced_schedule_on_random_graphs(kind):
    """Over random graphs of each family and round sizes from 1 to 1000: the balanced
    schedule is a permutation of the updates, keeps every dependency strictly earlier, has
    the as-early-as-possible level count, and never takes more kernel rounds than the
    as-early-as-possible schedule (on long chains with small rounds the fill alone can take
    one more; the as-early-as-possible levels are kept there)."""
    rng = np.random.default_rng({"sparse": 1, "tree": 2, "star": 3, "path": 4, "regular3": 5}[kind])
    for _ in range(24):
        n = int(rng.integers(2, 200))
        if kind == "regular3":
            n += n % 2
            n = max(n, 4)
        pairs = _random_graph(kind, n, rng)
        ei = np.array([a for a, _ in pairs], np.int32)
        ej = np.array([b for _, b in pairs], np.int32)
        _, off0 = pt.make_schedule(n, ei, ej)
        adj = [set() for _ in range(n)]
        for a, b in pairs:
            adj[a].add(b)
            adj[b].add(a)
        for k in (1, 2, 3, 4, 7, 8, 16, 32, 48, 96, 1000):
            items, off = pt.make_schedule(n, ei, ej, items_per_round=k)
            assert sorted(items.tolist()) == list(range(2 * n))
            assert off.size == off0.size
            level = _levels(items, off)
            for i in range(n):
                assert level[2 * i] < level[2 * i + 1]
                for j in adj[i]:
                    if j < i:
                        assert level[2 * j] < level[2 * i] and level[2 * j + 1] < level[2 * i + 1]
            assert _rounds(off, k) <= _rounds(off0, k), (kind, n, k)
