"""ctypes binding of pt_mt.c: the paper's multi-threaded CPU Parallel Tempering (Sec. 4,
Figs. 4-5) -- persistent threads, a work pool of chains handed out hardest first, explicit
barriers and a parallel swap pass.

A CPU comparison baseline for the benchmark. The GPU library never loads it (it has no CPU
fallback), and it is not the oracle the tests trust: its results are checked against the
oracle like the GPU path's.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pt_mt.c")
HDR = os.path.join(HERE, "pt_mt.h")
LIB = os.path.join(HERE, "libcpupt.so")
CFLAGS = ["-O3", "-fPIC", "-shared", "-pthread", "-std=c11", "-ffp-contract=off"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    stale = not os.path.exists(LIB) or any(os.path.getmtime(f) > os.path.getmtime(LIB) for f in (SRC, HDR))
    if force or stale:
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", *CFLAGS, "-I", HERE, "-o", tmp, SRC, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            lib.cpt_create.argtypes = [i32, i32, vp, vp, vp, vp, i32, i32, vp, vp, u64, i32]
            lib.cpt_create.restype = vp
            lib.cpt_run.argtypes = [vp, i64, i32]
            lib.cpt_read_state.argtypes = [vp, vp]
            lib.cpt_read_obs.argtypes = [vp] * 13
            lib.cpt_destroy.argtypes = [vp]
            lib.cpt_lmax.argtypes = [vp]
            lib.cpt_lmax.restype = i32
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class CpuPT:
    """One PT-QMC problem on the host cores. thr and coef are the Metropolis thresholds
    [R][2 Lmax + 1][3] and swap coefficients [2 (R - 1)] (the same tables the GPU library
    and the oracle build from the ladder)."""

    def __init__(self, prob, thr, coef, threads=None):
        self.lib = load()
        self.N, self.P, self.R = int(prob.n), int(prob.P), int(prob.R)
        self._keep = [np.ascontiguousarray(a, np.int32) for a in (prob.ei, prob.ej, prob.J, prob.h)]
        self._thr = np.ascontiguousarray(thr, np.uint32)
        self._coef = np.ascontiguousarray(coef if np.size(coef) else np.zeros(2), np.float64)
        self.threads = int(threads or os.cpu_count() or 1)
        self.h = self.lib.cpt_create(self.N, int(self._keep[0].size), *(_ptr(a) for a in self._keep), self.P, self.R,
                                     _ptr(self._thr), _ptr(self._coef), int(prob.seed) & 0xFFFFFFFFFFFFFFFF,
                                     self.threads)
        if not self.h:
            raise ValueError("cpt_create rejected the problem")
        lmax = self.lib.cpt_lmax(self.h)
        if self._thr.size != self.R * (2 * lmax + 1) * 3:
            self.close()
            raise ValueError("threshold table has %d entries, need R*(2*%d+1)*3" % (self._thr.size, lmax))

    @classmethod
    def from_problem(cls, prob, threads=None):
        """Tables from the oracle-independent host helper of the GPU library (data only)."""
        from paper_1004_0023_gb300 import pt

        lmax = _lmax(prob)
        thr, coef = pt.make_tables(prob.P, prob.T, prob.gamma, lmax)
        return cls(prob, thr, coef, threads)

    def run(self, n_sweeps, sweeps_per_swap):
        self.lib.cpt_run(self.h, int(n_sweeps), int(sweeps_per_swap))

    def read_state(self):
        out = np.empty((self.R, self.N, self.P), np.int8)
        self.lib.cpt_read_state(self.h, _ptr(out))
        return out

    def obs(self):
        R = self.R
        tq = np.zeros(2, np.int64)
        arr = {k: np.zeros(R, np.int64) for k in ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc")}
        att = np.zeros(max(R, 1), np.int64)
        acc = np.zeros(max(R, 1), np.int64)
        at = np.zeros(R, np.int32)
        self.lib.cpt_read_obs(self.h, _ptr(tq), *(_ptr(arr[k]) for k in
                                                  ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2",
                                                   "flip_acc")), _ptr(att), _ptr(acc), _ptr(at))
        d = dict(arr)
        d["t"], d["q"] = int(tq[0]), int(tq[1])
        d["swap_att"], d["swap_acc"] = att[: R - 1], acc[: R - 1]
        d["replica_at"] = at
        return d

    def close(self):
        if getattr(self, "h", None):
            self.lib.cpt_destroy(self.h)
            self.h = None

    __del__ = close


def _lmax(prob):
    lm = np.abs(np.asarray(prob.h, np.int64)).copy()
    for a, b, J in zip(prob.ei, prob.ej, prob.J):
        lm[a] += abs(int(J))
        lm[b] += abs(int(J))
    return int(lm.max()) if lm.size else 0
