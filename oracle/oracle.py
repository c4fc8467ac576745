"""ctypes wrapper around the plain C oracle (oracle/pt_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg of the
benchmark are the only users. The product library never imports this module, and this
module imports nothing from the product package. It takes plain arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pt_oracle.c")
HDR = os.path.join(HERE, "pt_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = ["-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp", "-std=c11"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    """Compile the oracle with gcc (plain C, no FP contraction). Returns the library path."""
    stale = (not os.path.exists(out)) or any(
        os.path.getmtime(f) > os.path.getmtime(out) for f in (src, HDR)
    )
    if force or stale:
        tmp = out + ".tmp%d" % os.getpid()
        cmd = ["gcc", *CFLAGS, "-I", HERE, "-o", tmp, src, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _declare(lib):
    i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.orc_philox.argtypes = [vp, vp, vp]
    lib.orc_det_exp.argtypes = [dbl]
    lib.orc_det_exp.restype = dbl
    lib.orc_det_exp_array.argtypes = [vp, vp, i64]
    lib.orc_create.argtypes = [i32, i32, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, u64]
    lib.orc_create.restype = vp
    lib.orc_error.restype = ctypes.c_char_p
    lib.orc_destroy.argtypes = [vp]
    lib.orc_set_threads.argtypes = [vp, i32]
    lib.orc_lmax.argtypes = [vp]
    lib.orc_lmax.restype = i32
    lib.orc_flip_table.argtypes = [vp, vp]
    lib.orc_swap_coef.argtypes = [vp, vp]
    lib.orc_sweep.argtypes = [vp, i64]
    lib.orc_swap.argtypes = [vp]
    lib.orc_run.argtypes = [vp, i64, i32]
    lib.orc_read_state.argtypes = [vp, vp]
    lib.orc_read_replica_state.argtypes = [vp, vp]
    lib.orc_write_state.argtypes = [vp, vp]
    lib.orc_write_state.restype = ctypes.c_int
    lib.orc_read_obs.argtypes = [vp] * 13


def load(path: str | None = None):
    """Load (building first if needed) the oracle library. A path loads a private copy."""
    global _lib
    if path is not None:
        lib = ctypes.CDLL(path)
        _declare(lib)
        return lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            _declare(lib)
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key, lib=None) -> np.ndarray:
    lib = lib or load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def det_exp(x, lib=None) -> np.ndarray:
    lib = lib or load()
    xa = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(xa)
    lib.orc_det_exp_array(_ptr(xa), _ptr(y), xa.size)
    return y


class Oracle:
    """One PT-QMC problem (instance + Trotter slices + ladder + seed) run on the CPU."""

    def __init__(self, n, ei, ej, J, h, P, T, gamma, seed, flip_thr=None, swap_coef=None,
                 threads=1, lib=None):
        self.lib = lib or load()
        self.N, self.P = int(n), int(P)
        self._ei = np.ascontiguousarray(ei, np.int32)
        self._ej = np.ascontiguousarray(ej, np.int32)
        self._J = np.ascontiguousarray(J, np.int32)
        self._h = np.ascontiguousarray(h, np.int32)
        self._T = np.ascontiguousarray(T, np.float64)
        self._g = np.ascontiguousarray(gamma, np.float64)
        self.R = int(self._T.size)
        thr = None if flip_thr is None else np.ascontiguousarray(flip_thr, np.uint32)
        coef = None if swap_coef is None else np.ascontiguousarray(swap_coef, np.float64)
        self._h_ptr = self.lib.orc_create(
            self.N, int(self._ei.size), _ptr(self._ei), _ptr(self._ej), _ptr(self._J), _ptr(self._h),
            self.P, self.R, _ptr(self._T), _ptr(self._g),
            None if thr is None else _ptr(thr), None if coef is None else _ptr(coef),
            ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF))
        if not self._h_ptr:
            raise ValueError("oracle rejected the problem: " + self.lib.orc_error().decode())
        self.lmax = int(self.lib.orc_lmax(self._h_ptr))
        if threads != 1:
            self.lib.orc_set_threads(self._h_ptr, int(threads))

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.n, prob.ei, prob.ej, prob.J, prob.h, prob.P, prob.T, prob.gamma,
                   prob.seed, **kw)

    def close(self):
        if getattr(self, "_h_ptr", None):
            self.lib.orc_destroy(self._h_ptr)
            self._h_ptr = None

    __del__ = close

    def flip_table(self) -> np.ndarray:
        out = np.zeros((self.R, 2 * self.lmax + 1, 3), np.uint32)
        self.lib.orc_flip_table(self._h_ptr, _ptr(out))
        return out

    def swap_coef(self) -> np.ndarray:
        out = np.zeros(2 * max(self.R - 1, 0), np.float64)
        if out.size:
            self.lib.orc_swap_coef(self._h_ptr, _ptr(out))
        return out

    def sweep(self, n: int = 1):
        self.lib.orc_sweep(self._h_ptr, int(n))

    def swap(self):
        self.lib.orc_swap(self._h_ptr)

    def run(self, n_sweeps: int, sweeps_per_swap: int):
        self.lib.orc_run(self._h_ptr, int(n_sweeps), int(sweeps_per_swap))

    def read_state(self) -> np.ndarray:
        out = np.zeros((self.R, self.N, self.P), np.int8)
        self.lib.orc_read_state(self._h_ptr, _ptr(out))
        return out

    def read_replica_state(self) -> np.ndarray:
        out = np.zeros((self.R, self.N, self.P), np.int8)
        self.lib.orc_read_replica_state(self._h_ptr, _ptr(out))
        return out

    def write_state(self, x: np.ndarray):
        xa = np.ascontiguousarray(x, np.int8)
        assert xa.shape == (self.R, self.N, self.P)
        if self.lib.orc_write_state(self._h_ptr, _ptr(xa)) != 0:
            raise ValueError("spins must be +1 or -1")

    def obs(self) -> dict:
        R = self.R
        tq = np.zeros(2, np.int64)
        per_rung = {k: np.zeros(R, np.int64) for k in
                    ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc")}
        att = np.zeros(max(R - 1, 1), np.int64)
        acc = np.zeros(max(R - 1, 1), np.int64)
        at = np.zeros(R, np.int32)
        self.lib.orc_read_obs(self._h_ptr, _ptr(tq), *(_ptr(per_rung[k]) for k in
                              ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc")),
                              _ptr(att), _ptr(acc), _ptr(at))
        d = dict(per_rung)
        d["t"], d["q"] = int(tq[0]), int(tq[1])
        d["swap_att"], d["swap_acc"] = att[: R - 1], acc[: R - 1]
        d["replica_at"] = at
        return d
