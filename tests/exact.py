"""Exact references the oracle is pinned to (independent of the oracle's code).

- ``enumerate_st``: the Suzuki-Trotter (ST) Boltzmann distribution exp(-S_r(X)) by
  listing all 2^(N*P) states (tiny systems).
- ``transfer_matrix``: the same moments for N <= 10 at any P from Z = Tr T^P.
- ``exact_diag``: the thermal energy of H = sum J Z Z + sum h Z - Gamma sum X by full
  diagonalisation, and ``st_energy_estimator`` which maps ST moments to <H>.

The ST mapping (Sec. 6 connects many copies of the classical system; the copies are
coupled through K = -1/2 ln tanh(beta Gamma / P)) is cross-checked here against
quantum mechanics by ``exact_diag``, so the formula is not only retyped.
"""
from __future__ import annotations

import itertools

import numpy as np


def slice_energies(n, ei, ej, J, h):
    """E(s) for all 2^n single-copy states; state code bit i set => s_i = -1."""
    codes = np.arange(2 ** n)
    s = 1 - 2 * ((codes[:, None] >> np.arange(n)[None, :]) & 1)  # [2^n, n]
    E = (s[:, ei] * s[:, ej] * np.asarray(J)[None, :]).sum(1) + (s * np.asarray(h)[None, :]).sum(1)
    return s, E.astype(np.float64)


def coupling(beta, gamma, P):
    a = beta * gamma / P
    return -0.5 * np.log(np.tanh(a))


def enumerate_st(prob, r):
    """Exact moments and state distribution of exp(-S_r) over all N*P spins."""
    n, P = prob.n, prob.P
    beta = 1.0 / prob.T[r]
    K = coupling(beta, prob.gamma[r], P)
    nbits = n * P
    assert nbits <= 20
    codes = np.arange(2 ** nbits, dtype=np.int64)
    # spin (i, k) is bit i*P + k
    bits = (codes[:, None] >> np.arange(nbits)[None, :]) & 1
    s = (1 - 2 * bits).reshape(-1, n, P).astype(np.int64)
    Ek = (s[:, prob.ei, :] * s[:, prob.ej, :] * prob.J[None, :, None]).sum(1) + (
        s * prob.h[None, :, None]).sum(1)
    Etot = Ek.sum(1).astype(np.float64)
    M = (s * np.roll(s, -1, axis=2)).sum((1, 2)).astype(np.float64)
    logw = -(beta / P) * Etot + K * M
    w = np.exp(logw - logw.max())
    w /= w.sum()
    return dict(E=float(w @ Etot), M=float(w @ M), E2=float(w @ Etot ** 2), M2=float(w @ M ** 2),
                prob=w, Etot=Etot, Mtot=M)


def state_code(x):
    """Code of one chain state x[n, P] in the bit order used by ``enumerate_st``."""
    flat = (np.asarray(x).reshape(-1) < 0).astype(np.int64)
    return int((flat << np.arange(flat.size)).sum())


def transfer_matrix(prob, r, P=None):
    """Exact <sum_k E(s^k)>, <M> of the ST system at rung r via Z = Tr T^P."""
    n = prob.n
    P = prob.P if P is None else P
    beta = 1.0 / prob.T[r]
    K = coupling(beta, prob.gamma[r], P)
    s, E = slice_energies(n, prob.ei, prob.ej, prob.J, prob.h)
    C = (s @ s.T).astype(np.float64)
    b = beta / P
    # symmetric transfer matrix T = D^1/2 exp(K C) D^1/2 with D = diag(exp(-b E))
    half = np.exp(-0.5 * b * (E - E.min()))
    logT = K * C
    shift = logT.max()
    T = half[:, None] * np.exp(logT - shift) * half[None, :]
    TC = T * C
    evals, V = np.linalg.eigh(T)
    lam = evals / np.abs(evals).max()

    def power(k):
        return (V * lam ** k) @ V.T

    TP = power(P)
    Z = np.trace(TP)
    Emean = P * float(np.sum(E * np.diag(TP))) / Z
    TPm1 = power(P - 1)
    # T^(P-1) in units where T is divided by max|eig|; TC uses the same scale
    scale = np.abs(evals).max()
    Mmean = P * float(np.trace(TPm1 @ (TC / scale))) / Z
    return dict(E=Emean, M=Mmean)


def exact_diag(prob, r):
    """Thermal <H> of the transverse-field Hamiltonian at rung r (2^N dense)."""
    n = prob.n
    beta = 1.0 / prob.T[r]
    g = prob.gamma[r]
    s, E = slice_energies(n, prob.ei, prob.ej, prob.J, prob.h)
    dim = 2 ** n
    H = np.diag(E)
    codes = np.arange(dim)
    for i in range(n):
        H[codes, codes ^ (1 << i)] += -g
    w = np.linalg.eigvalsh(H)
    p = np.exp(-beta * (w - w.min()))
    return float((w * p).sum() / p.sum())


def st_energy_estimator(Emean, Mmean, n, P, beta, gamma):
    """<H> from ST moments: -d ln Z_P / d beta with Z_P = (sinh(2a)/2)^(NP/2) sum exp(-S)."""
    a = beta * gamma / P
    return Emean / P - n * gamma / np.tanh(2 * a) + gamma * Mmean / (P * np.sinh(2 * a))


def batch_means(samples_fn, n_batches, per_batch):
    """Runs n_batches; samples_fn(per_batch) returns per-rung batch means; returns mean, SE."""
    bm = np.asarray([samples_fn(per_batch) for _ in range(n_batches)], np.float64)
    return bm.mean(0), bm.std(0, ddof=1) / np.sqrt(n_batches)


def all_states(n):
    return list(itertools.product((1, -1), repeat=n))
