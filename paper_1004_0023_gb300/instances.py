"""Seeded synthetic PT-QMC problems (inputs only; no part of the method's arithmetic).

The paper's own problems (AQUA Ising instances of 8-96 qubits, 128 Trotter copies,
27-111 chains; Sec. 6, Table 1) are not public. These generators stand in for them with
the shapes named by the workloads below: sparse random graphs with small integer
couplings, a ladder of transverse fields at fixed temperature, and a Philox seed.

Both the CUDA library and the CPU oracle consume these arrays; this module computes no
acceptance probability, energy or random draw of the method.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    """One PT-QMC problem: an N-site Ising instance, P Trotter copies, R rungs, a seed."""

    n: int
    ei: np.ndarray          # int32[n_edges]
    ej: np.ndarray          # int32[n_edges]
    J: np.ndarray           # int32[n_edges], non-zero
    h: np.ndarray           # int32[n]
    P: int
    T: np.ndarray           # float64[R]
    gamma: np.ndarray       # float64[R]
    seed: int               # Philox key (64 bit)
    n_sweeps: int = 0
    sweeps_per_swap: int = 1
    name: str = ""

    @property
    def R(self) -> int:
        return int(self.T.size)

    @property
    def attempts_per_sweep(self) -> int:
        return self.n * self.P * self.R


def random_regular_graph(n: int, d: int, rng: np.random.Generator):
    """Uniform simple d-regular graph by the pairing model with rejection."""
    if (n * d) % 2 or d >= n:
        raise ValueError("need n*d even and d < n")
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    for _ in range(10000):
        perm = rng.permutation(stubs)
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        key = lo * n + hi
        if np.unique(key).size != key.size:
            continue
        order = np.argsort(key)
        return lo[order].astype(np.int32), hi[order].astype(np.int32)
    raise RuntimeError("pairing model did not produce a simple graph")


def chimera_graph(rows: int, cols: int):
    """K4,4 unit cells on a rows x cols grid (8 sites per cell).

    Within a cell every site of shore A (local 0-3) couples to every site of shore B
    (local 4-7). Shore-A site l couples to site l of the cell below, shore-B site l to
    site l of the cell to the right: degree 6 inside the grid, 5 on its edge.
    """
    ei, ej = [], []
    for r in range(rows):
        for c in range(cols):
            base = 8 * (r * cols + c)
            for a in range(4):
                for b in range(4, 8):
                    ei.append(base + a)
                    ej.append(base + b)
            if r + 1 < rows:
                below = 8 * ((r + 1) * cols + c)
                for a in range(4):
                    ei.append(base + a)
                    ej.append(below + a)
            if c + 1 < cols:
                right = 8 * (r * cols + c + 1)
                for b in range(4, 8):
                    ei.append(base + b)
                    ej.append(right + b)
    return np.asarray(ei, np.int32), np.asarray(ej, np.int32)


def gamma_ladder(kind: str, g0: float, g1: float, R: int) -> np.ndarray:
    if R == 1:
        return np.asarray([g0], np.float64)
    if kind == "linear":
        return np.asarray([g0 + (g1 - g0) * r / (R - 1) for r in range(R)], np.float64)
    if kind == "geometric":
        return np.asarray([g0 * (g1 / g0) ** (r / (R - 1)) for r in range(R)], np.float64)
    raise ValueError(kind)


def _draw(values, size, rng):
    return np.asarray(values, np.int32)[rng.integers(0, len(values), size=size)]


def philox_seed(index: int) -> int:
    return 0x5EED0000 + int(index)


# Workloads (sizes as in the problem statement of this library's benchmark).
WORKLOADS = {
    # random 3-regular, N=16, P=32, R=16, linear Gamma 0.1..3.0 at T=0.05, 10^4 sweeps
    "regular3_n16_p32_r16": dict(graph="regular", n=16, degree=3, J=(-2, -1, 1, 2), h=(-1, 0, 1),
                                 P=32, R=16, ladder="linear", g0=0.1, g1=3.0, T=0.05,
                                 n_sweeps=10000),
    # random 3-regular, N=256, P=64, R=64, geometric Gamma 0.05..4.0 at T=0.02, 2000 sweeps
    "regular3_n256_p64_r64": dict(graph="regular", n=256, degree=3, J=(-2, -1, 1, 2), h=(-1, 0, 1),
                                  P=64, R=64, ladder="geometric", g0=0.05, g1=4.0, T=0.02,
                                  n_sweeps=2000),
    # K4,4 cells on a 16x16 grid (N=2048), J in {-4..4}\{0}, h=0, P=128, R=96, 500 sweeps.
    # The ladder is not stated for this size; geometric Gamma 0.05..4.0 at T=0.02 is used.
    "chimera16_n2048_p128_r96": dict(graph="chimera", rows=16, cols=16,
                                     J=(-4, -3, -2, -1, 1, 2, 3, 4), h=(0,), P=128, R=96,
                                     ladder="geometric", g0=0.05, g1=4.0, T=0.02, n_sweeps=500),
    # classical parallel tempering (P = 1, Gamma = 0) on the N=256 graph family: R=64
    # temperatures geometric 0.1..3.0, 2000 sweeps, one swap pass per sweep
    "classical_regular3_n256_r64": dict(graph="regular", n=256, degree=3, J=(-2, -1, 1, 2), h=(-1, 0, 1),
                                        P=1, R=64, ladder="temperature", g0=0.1, g1=3.0, n_sweeps=2000),
}


def make_problem(graph: str, rng: np.random.Generator, *, n=None, degree=3, rows=None, cols=None,
                 J=(-2, -1, 1, 2), h=(-1, 0, 1), P=32, R=16, ladder="geometric", g0=0.05, g1=4.0,
                 T=0.02, n_sweeps=0, sweeps_per_swap=1, seed=0, name="") -> Problem:
    if graph == "regular":
        ei, ej = random_regular_graph(int(n), int(degree), rng)
        nn = int(n)
    elif graph == "chimera":
        ei, ej = chimera_graph(int(rows), int(cols))
        nn = 8 * int(rows) * int(cols)
    else:
        raise ValueError(graph)
    Jv = _draw(J, ei.size, rng)
    hv = _draw(h, nn, rng)
    if ladder == "temperature":
        # classical parallel tempering (P = 1): geometric temperatures g0..g1, Gamma = 0
        Tv = gamma_ladder("geometric", g0, g1, int(R))
        gam = np.zeros(int(R), np.float64)
    else:
        gam = gamma_ladder(ladder, g0, g1, int(R))
        Tv = np.full(int(R), float(T), np.float64)
    return Problem(nn, ei, ej, Jv, hv, int(P), Tv, gam, int(seed), int(n_sweeps),
                   int(sweeps_per_swap), name)


def workload(name: str, index: int = 1) -> Problem:
    """A named workload drawn with generator seed `index` and Philox seed 0x5EED0000+index."""
    spec = dict(WORKLOADS[name])
    rng = np.random.default_rng(index)
    return make_problem(spec.pop("graph"), rng, seed=philox_seed(index), name=name, **spec)


def batch_problems(count: int = 512, index: int = 1, n_sweeps: int = 1000,
                   p_choices=(32, 64, 128), n_range=(32, 1024), r_range=(16, 128)):
    """Independent problems of uneven size for one batched launch.

    N ~ U{32..1024}; the graph is random 3-regular or a K4,4 cell lattice of degree <= 6
    (N rounded down to whole cells); P ~ U{32,64,128}; R ~ U{16..128}; J in {-2,-1,1,2},
    h in {-1,0,1}; geometric Gamma 0.05..4.0 at T=0.02; one swap pass per sweep.
    """
    rng = np.random.default_rng(1_000_003 * index + 17)
    out = []
    for b in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        P = int(p_choices[int(rng.integers(0, len(p_choices)))])
        R = int(rng.integers(r_range[0], r_range[1] + 1))
        seed = philox_seed(index * 100000 + b)
        if rng.integers(0, 2) == 0:
            n += n % 2
            prob = make_problem("regular", rng, n=n, degree=3, P=P, R=R, n_sweeps=n_sweeps,
                                seed=seed, name="batch%d" % b)
        else:
            cells = max(1, n // 8)
            rows = max(1, int(math.isqrt(cells)))
            cols = max(1, cells // rows)
            prob = make_problem("chimera", rng, rows=rows, cols=cols, P=P, R=R,
                                n_sweeps=n_sweeps, seed=seed, name="batch%d" % b)
        out.append(prob)
    return out


def tiny_problem(n, edges, J, h, P, T, gamma, seed=1, name="tiny") -> Problem:
    """A hand-specified problem (used by the exact-enumeration checks)."""
    e = np.asarray(edges, np.int64).reshape(-1, 2)
    return Problem(int(n), e[:, 0].astype(np.int32), e[:, 1].astype(np.int32),
                   np.asarray(J, np.int32), np.asarray(h, np.int32), int(P),
                   np.asarray(T, np.float64), np.asarray(gamma, np.float64), int(seed), 0, 1, name)
