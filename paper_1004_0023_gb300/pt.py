"""Thin ctypes binding of the C ABI in include/pt.h (argument marshalling only).

Every step of the PT-QMC path runs in the CUDA kernels of ``libpt.so``; this module only
converts numpy arrays to pointers and back. There is no CPU fallback: if the library is
missing, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpt.so")

PT_OK, PT_EINVAL, PT_ENOMEM, PT_ECUDA, PT_EOVERFLOW, PT_ETIMEDOUT, PT_EBUSY, PT_ENODEV = (
    0, -1, -2, -3, -4, -5, -6, -7)
# fixed swap-mailbox entries of pt_run_noalloc (PT_NOALLOC_MAILBOXES in include/pt.h)
PT_NOALLOC_MAILBOXES = 16384
_NAMES = {0: "PT_OK", -1: "PT_EINVAL", -2: "PT_ENOMEM", -3: "PT_ECUDA", -4: "PT_EOVERFLOW",
          -5: "PT_ETIMEDOUT", -6: "PT_EBUSY", -7: "PT_ENODEV"}

_i32, _i64, _u64, _dbl, _vp, _sz = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_void_p, ctypes.c_size_t)
_p_i32, _p_i64 = ctypes.POINTER(_i32), ctypes.POINTER(_i64)


class pt_instance(ctypes.Structure):
    _fields_ = [("n", _i32), ("n_edges", _i32), ("ei", _p_i32), ("ej", _p_i32), ("J", _p_i32),
                ("h", _p_i32)]


class pt_rung(ctypes.Structure):
    _fields_ = [("T", _dbl), ("gamma", _dbl)]


class pt_options(ctypes.Structure):
    _fields_ = [("threads_per_block", _i32), ("wait_timeout_ms", _i32), ("swap_mode", _i32),
                ("test_withhold_rung", _i32), ("kernel_path", _i32), ("producer_threads", _i32),
                ("test_exact_swaps", _i32), ("cluster_size", _i32), ("no_autotune", _i32), ("group_threads", _i32),
                ("reserved", _i32 * 2)]


class pt_observables(ctypes.Structure):
    _fields_ = [("t", _i64), ("q", _i64), ("E", _p_i64), ("M", _p_i64), ("n_meas", _p_i64),
                ("sum_E", _p_i64), ("sum_E2", _p_i64), ("sum_M", _p_i64), ("sum_M2", _p_i64),
                ("flip_acc", _p_i64), ("swap_att", _p_i64), ("swap_acc", _p_i64),
                ("replica_at", _p_i32)]


class pt_info(ctypes.Structure):
    _fields_ = [("n", _i32), ("P", _i32), ("R", _i32), ("lmax", _i32), ("max_degree", _i32),
                ("n_levels", _i32), ("threads_per_block", _i32), ("cooperative", _i32),
                ("kernel_path", _i32), ("producer_threads", _i32), ("device_bytes", _i64), ("kernel_launches", _i64),
                ("h2d_bytes", _i64), ("tuned_plans", _i32), ("reserved", _i32)]


class pt_request(ctypes.Structure):
    _fields_ = [("inst", pt_instance), ("P", _i32), ("ladder", ctypes.POINTER(pt_rung)), ("R", _i32),
                ("seed", _u64), ("n_sweeps", _i64), ("sweeps_per_swap", _i32)]


class pt_batch_info(ctypes.Structure):
    _fields_ = [("count", _i32), ("cluster", _i32), ("n_clusters", _i32), ("threads_per_block", _i32),
                ("smem_bytes", _i64), ("device_bytes", _i64), ("kernel_launches", _i64), ("h2d_bytes", _i64),
                ("tuned_layouts", _i32), ("group_widen", _i32), ("graph", _i32), ("reserved", _i32)]


class pt_server_options(ctypes.Structure):
    _fields_ = [("arena_bytes", _i64), ("max_active", _i32), ("quantum_sweeps", _i32), ("cluster_size", _i32),
                ("reserved", _i32 * 3)]


class pt_server_info(ctypes.Structure):
    _fields_ = [("active", _i32), ("queued", _i32), ("arena_bytes", _i64), ("arena_used", _i64), ("steps", _i64),
                ("kernel_launches", _i64), ("wide_steps", _i64), ("group_launches", _i64)]


class pt_device_problem(ctypes.Structure):
    _fields_ = [("n", _i32), ("P", _i32), ("R", _i32), ("lmax", _i32), ("row_stride", _i32), ("n_levels", _i32),
                ("nbr", _vp), ("h", _vp), ("items", _vp), ("level_off", _vp), ("thr", _vp), ("coef", _vp),
                ("spins", _vp), ("E", _vp), ("M", _vp), ("rung_of_slot", _vp), ("slot_of_rung", _vp),
                ("stats", _vp), ("swap_stats", _vp), ("status", _vp), ("seed", _u64), ("t0", _i64), ("q0", _i64)]


class PTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_NAMES.get(code, code), msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libpt.so (built by ``paper_1004_0023_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libpt.so is not built (%s); run paper_1004_0023_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    lib.pt_create.argtypes = [ctypes.POINTER(pt_instance), _i32, ctypes.POINTER(pt_rung), _i32, _vp, _vp,
                              _u64, ctypes.POINTER(pt_options), _vp, ctypes.POINTER(_vp)]
    lib.pt_sweep.argtypes = [_vp, _i64]
    lib.pt_swap.argtypes = [_vp]
    lib.pt_run.argtypes = [_vp, _i64, _i32]
    lib.pt_read_state.argtypes = [_vp, _vp, _sz]
    lib.pt_write_state.argtypes = [_vp, _vp, _sz]
    lib.pt_read_observables.argtypes = [_vp, ctypes.POINTER(pt_observables)]
    lib.pt_restore.argtypes = [_vp, _vp, _sz, ctypes.POINTER(pt_observables)]
    lib.pt_read_tables.argtypes = [_vp, _vp, _sz, _vp, _sz]
    lib.pt_get_info.argtypes = [_vp, ctypes.POINTER(pt_info)]
    lib.pt_sync.argtypes = [_vp]
    lib.pt_destroy.argtypes = [_vp]
    lib.pt_last_error.argtypes = [_vp]
    lib.pt_last_error.restype = ctypes.c_char_p
    lib.pt_make_tables.argtypes = [_i32, ctypes.POINTER(pt_rung), _i32, _i32, _vp, _vp]
    lib.pt_make_schedule.argtypes = [ctypes.POINTER(pt_instance), _vp, _vp, _p_i32]
    lib.pt_make_schedule_balanced.argtypes = [ctypes.POINTER(pt_instance), _i32, _vp, _vp, _p_i32]
    lib.pt_run_noalloc.argtypes = [ctypes.POINTER(pt_device_problem), _i64, _i32, _i32, _vp]
    lib.pt_batch_create.argtypes = [ctypes.POINTER(pt_request), _i32, ctypes.POINTER(pt_options), _vp,
                                    ctypes.POINTER(_vp)]
    lib.pt_batch_run.argtypes = [_vp]
    lib.pt_batch_sync.argtypes = [_vp]
    lib.pt_batch_read_state.argtypes = [_vp, _i32, _vp, _sz]
    lib.pt_batch_read_observables.argtypes = [_vp, _i32, ctypes.POINTER(pt_observables)]
    lib.pt_batch_get_info.argtypes = [_vp, ctypes.POINTER(pt_batch_info)]
    lib.pt_batch_destroy.argtypes = [_vp]
    lib.pt_batch_last_error.argtypes = [_vp]
    lib.pt_batch_last_error.restype = ctypes.c_char_p
    lib.pt_server_create.argtypes = [ctypes.POINTER(pt_server_options), _vp, ctypes.POINTER(_vp)]
    lib.pt_server_submit.argtypes = [_vp, ctypes.POINTER(pt_request), _p_i64]
    lib.pt_server_step.argtypes = [_vp, _p_i64, _i32, _p_i32]
    lib.pt_server_read_result.argtypes = [_vp, _i64, _vp, _sz, ctypes.POINTER(pt_observables)]
    lib.pt_server_release.argtypes = [_vp, _i64]
    lib.pt_server_get_info.argtypes = [_vp, ctypes.POINTER(pt_server_info)]
    lib.pt_server_destroy.argtypes = [_vp]
    lib.pt_server_last_error.argtypes = [_vp]
    lib.pt_server_last_error.restype = ctypes.c_char_p
    lib.pt_noalloc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def exported_symbols():
    """Names of the entry points declared in include/pt.h."""
    return ["pt_create", "pt_sweep", "pt_swap", "pt_run", "pt_read_state", "pt_write_state",
            "pt_read_observables", "pt_read_tables", "pt_get_info", "pt_sync", "pt_destroy",
            "pt_last_error", "pt_make_tables", "pt_make_schedule", "pt_make_schedule_balanced", "pt_run_noalloc",
            "pt_noalloc_last_error", "pt_batch_create", "pt_batch_run", "pt_batch_read_state",
            "pt_batch_read_observables", "pt_batch_get_info", "pt_batch_sync", "pt_batch_destroy",
            "pt_batch_last_error", "pt_server_create", "pt_server_submit", "pt_server_step",
            "pt_server_read_result", "pt_server_release", "pt_server_get_info", "pt_server_destroy",
            "pt_server_last_error"]


def _instance(n, ei, ej, J, h, keep):
    arrs = [np.ascontiguousarray(a, np.int32) for a in (ei, ej, J, h)]
    keep.extend(arrs)
    return pt_instance(int(n), int(arrs[0].size), *(a.ctypes.data_as(_p_i32) for a in arrs))


def make_tables(P, T, gamma, lmax):
    """Host-only: the FP64 Metropolis thresholds and swap coefficients pt_create builds."""
    lib = load()
    T = np.asarray(T, np.float64)
    gamma = np.asarray(gamma, np.float64)
    R = int(T.size)
    ladder = (pt_rung * R)(*[pt_rung(float(a), float(b)) for a, b in zip(T, gamma)])
    thr = np.zeros((R, 2 * int(lmax) + 1, 3), np.uint32)
    coef = np.zeros(max(2 * (R - 1), 1), np.float64)
    rc = lib.pt_make_tables(int(P), ladder, R, int(lmax), _ptr(thr), _ptr(coef))
    if rc != PT_OK:
        raise PTError(rc, "pt_make_tables rejected its arguments")
    return thr, coef[: 2 * (R - 1)]


def make_schedule(n, ei, ej, items_per_round=0):
    """Host-only: the sweep's dependency-level schedule (items grouped by level); as early as
    possible, or balanced for a kernel taking items_per_round items of a level at a time."""
    lib = load()
    keep = []
    ei = np.asarray(ei, np.int32)
    inst = _instance(n, ei, ej, np.ones(ei.size, np.int32), np.zeros(int(n), np.int32), keep)
    items = np.zeros(2 * int(n), np.uint32)
    off = np.zeros(2 * int(n) + 1, np.int32)
    nlev = _i32()
    if items_per_round:
        rc = lib.pt_make_schedule_balanced(ctypes.byref(inst), int(items_per_round), _ptr(items), _ptr(off),
                                           ctypes.byref(nlev))
    else:
        rc = lib.pt_make_schedule(ctypes.byref(inst), _ptr(items), _ptr(off), ctypes.byref(nlev))
    if rc != PT_OK:
        raise PTError(rc, "pt_make_schedule rejected its arguments")
    return items, off[: nlev.value + 1]


def _ptr(a):
    return a.ctypes.data_as(_vp)


def run_noalloc(problem, n_sweeps, sweeps_per_swap, wait_timeout_ms=0, stream=None):
    """pt_run_noalloc on a filled pt_device_problem (device pointers owned by the caller)."""
    lib = load()
    rc = lib.pt_run_noalloc(ctypes.byref(problem), int(n_sweeps), int(sweeps_per_swap), int(wait_timeout_ms),
                            None if stream is None else _vp(int(stream)))
    if rc != PT_OK:
        raise PTError(rc, lib.pt_noalloc_last_error().decode())


class PT:
    """One PT-QMC context on the current CUDA device (see include/pt.h)."""

    def __init__(self, n, ei, ej, J, h, P, T, gamma, seed, flip_thr=None, swap_coef=None,
                 threads_per_block=0, wait_timeout_ms=0, swap_mode=0, stream=None,
                 test_withhold_rung=-1, kernel_path=0, producer_threads=0, test_exact_swaps=0, no_autotune=0,
                 cluster_size=0, group_threads=0):
        self.lib = load()
        self._arrays = [np.ascontiguousarray(a, np.int32) for a in (ei, ej, J, h)]
        inst = pt_instance(int(n), int(self._arrays[0].size),
                           *(a.ctypes.data_as(_p_i32) for a in self._arrays))
        T = np.asarray(T, np.float64)
        gamma = np.asarray(gamma, np.float64)
        self.N, self.P, self.R = int(n), int(P), int(T.size)
        ladder = (pt_rung * self.R)(*[pt_rung(float(a), float(b)) for a, b in zip(T, gamma)])
        thr = None if flip_thr is None else np.ascontiguousarray(flip_thr, np.uint32)
        coef = None if swap_coef is None else np.ascontiguousarray(swap_coef, np.float64)
        opt = pt_options(int(threads_per_block), int(wait_timeout_ms), int(swap_mode),
                         int(test_withhold_rung) + 1, int(kernel_path), int(producer_threads),
                         int(test_exact_swaps), int(cluster_size), int(no_autotune), int(group_threads))
        h_out = _vp()
        rc = self.lib.pt_create(ctypes.byref(inst), self.P, ladder, self.R,
                                None if thr is None else _ptr(thr), None if coef is None else _ptr(coef),
                                ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), ctypes.byref(opt),
                                None if stream is None else _vp(int(stream)), ctypes.byref(h_out))
        if rc != PT_OK:
            raise PTError(rc, self.lib.pt_last_error(None).decode())
        self.ctx = h_out
        self.info = self.get_info()

    @classmethod
    def from_problem(cls, prob, **kw):
        return cls(prob.n, prob.ei, prob.ej, prob.J, prob.h, prob.P, prob.T, prob.gamma, prob.seed, **kw)

    def _check(self, rc):
        if rc != PT_OK:
            raise PTError(rc, self.lib.pt_last_error(self.ctx).decode())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.pt_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sweep(self, n=1):
        self._check(self.lib.pt_sweep(self.ctx, int(n)))

    def swap(self):
        self._check(self.lib.pt_swap(self.ctx))

    def run(self, n_sweeps, sweeps_per_swap):
        self._check(self.lib.pt_run(self.ctx, int(n_sweeps), int(sweeps_per_swap)))

    def sync(self):
        self._check(self.lib.pt_sync(self.ctx))

    def read_state(self, out=None):
        if out is None:
            out = np.empty((self.R, self.N, self.P), np.int8)
        self._check(self.lib.pt_read_state(self.ctx, _ptr(out), out.nbytes))
        return out

    def write_state(self, x):
        xa = np.ascontiguousarray(x, np.int8)
        self._check(self.lib.pt_write_state(self.ctx, _ptr(xa), xa.nbytes))

    def obs(self):
        return _read_obs(self.R, lambda o: self.lib.pt_read_observables(self.ctx, ctypes.byref(o)), self._check)

    def checkpoint(self):
        """(state, observables) to hand to `restore` (pt_read_state + pt_read_observables)."""
        return self.read_state(), self.obs()

    def restore(self, state, obs):
        """pt_restore: continue bit for bit from a checkpoint of a context of the same problem."""
        xa = np.ascontiguousarray(state, np.int8)
        keep = {k: np.ascontiguousarray(obs[k], np.int64) for k in
                ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc")}
        att = np.zeros(max(self.R - 1, 1), np.int64)
        acc = np.zeros(max(self.R - 1, 1), np.int64)
        att[: self.R - 1] = obs["swap_att"]
        acc[: self.R - 1] = obs["swap_acc"]
        at = np.ascontiguousarray(obs["replica_at"], np.int32)
        o = pt_observables(int(obs["t"]), int(obs["q"]),
                           *(keep[k].ctypes.data_as(_p_i64) for k in
                             ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc")),
                           att.ctypes.data_as(_p_i64), acc.ctypes.data_as(_p_i64), at.ctypes.data_as(_p_i32))
        self._check(self.lib.pt_restore(self.ctx, _ptr(xa), xa.nbytes, ctypes.byref(o)))

    def tables(self):
        info = self.info
        thr = np.zeros((self.R, 2 * info.lmax + 1, 3), np.uint32)
        coef = np.zeros(max(2 * (self.R - 1), 1), np.float64)
        self._check(self.lib.pt_read_tables(self.ctx, _ptr(thr), thr.size, _ptr(coef), coef.size))
        return thr, coef[: 2 * (self.R - 1)]

    def get_info(self):
        i = pt_info()
        self._check(self.lib.pt_get_info(self.ctx, ctypes.byref(i)))
        return i


def _read_obs(R, call, check):
    arr = {k: np.zeros(R, np.int64) for k in
           ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc")}
    att = np.zeros(max(R - 1, 1), np.int64)
    acc = np.zeros(max(R - 1, 1), np.int64)
    at = np.zeros(R, np.int32)
    o = pt_observables(0, 0, *(arr[k].ctypes.data_as(_p_i64) for k in
                               ("E", "M", "n_meas", "sum_E", "sum_E2", "sum_M", "sum_M2", "flip_acc")),
                       att.ctypes.data_as(_p_i64), acc.ctypes.data_as(_p_i64), at.ctypes.data_as(_p_i32))
    check(call(o))
    d = dict(arr)
    d["t"], d["q"] = int(o.t), int(o.q)
    d["swap_att"], d["swap_acc"] = att[: R - 1], acc[: R - 1]
    d["replica_at"] = at
    return d


class Batch:
    """Many independent problems in one persistent launch (include/pt.h, pt_batch_*)."""

    def __init__(self, problems, cluster_size=0, stream=None):
        self.lib = load()
        self.problems = list(problems)
        keep = []
        reqs = (pt_request * len(self.problems))()
        for k, prob in enumerate(self.problems):
            inst = _instance(prob.n, prob.ei, prob.ej, prob.J, prob.h, keep)
            ladder = (pt_rung * prob.R)(*[pt_rung(float(a), float(b)) for a, b in zip(prob.T, prob.gamma)])
            keep.append(ladder)
            reqs[k] = pt_request(inst, int(prob.P), ladder, int(prob.R),
                                 int(prob.seed) & 0xFFFFFFFFFFFFFFFF, int(prob.n_sweeps), int(prob.sweeps_per_swap))
        opt = pt_options()
        opt.cluster_size = int(cluster_size)
        h = _vp()
        rc = self.lib.pt_batch_create(reqs, len(self.problems), ctypes.byref(opt),
                                      None if stream is None else _vp(int(stream)), ctypes.byref(h))
        if rc != PT_OK:
            raise PTError(rc, self.lib.pt_batch_last_error(None).decode())
        self.handle = h

    def _check(self, rc):
        if rc != PT_OK:
            raise PTError(rc, self.lib.pt_batch_last_error(self.handle).decode())

    def run(self):
        self._check(self.lib.pt_batch_run(self.handle))

    def sync(self):
        self._check(self.lib.pt_batch_sync(self.handle))

    def read_state(self, k, out=None):
        prob = self.problems[k]
        if out is None:
            out = np.empty((prob.R, prob.n, prob.P), np.int8)
        self._check(self.lib.pt_batch_read_state(self.handle, int(k), _ptr(out), out.nbytes))
        return out

    def obs(self, k):
        return _read_obs(self.problems[k].R,
                         lambda o: self.lib.pt_batch_read_observables(self.handle, int(k), ctypes.byref(o)),
                         self._check)

    def info(self):
        i = pt_batch_info()
        self._check(self.lib.pt_batch_get_info(self.handle, ctypes.byref(i)))
        return i

    def close(self):
        if getattr(self, "handle", None):
            self.lib.pt_batch_destroy(self.handle)
            self.handle = None

    __del__ = close


def _request(prob, keep):
    inst = _instance(prob.n, prob.ei, prob.ej, prob.J, prob.h, keep)
    ladder = (pt_rung * prob.R)(*[pt_rung(float(a), float(b)) for a, b in zip(prob.T, prob.gamma)])
    keep.append(ladder)
    return pt_request(inst, int(prob.P), ladder, int(prob.R), int(prob.seed) & 0xFFFFFFFFFFFFFFFF,
                      int(prob.n_sweeps), int(prob.sweeps_per_swap))


class Server:
    """Continuous-batching server (include/pt.h, pt_server_*)."""

    def __init__(self, arena_bytes=0, max_active=0, quantum_sweeps=0, cluster_size=0, stream=None,
                 stepped=False, packed_only=False):
        self.lib = load()
        opt = pt_server_options(int(arena_bytes), int(max_active), int(quantum_sweeps), int(cluster_size))
        opt.reserved[0] = 1 if packed_only else 0
        opt.reserved[1] = 1 if stepped else 0
        h = _vp()
        rc = self.lib.pt_server_create(ctypes.byref(opt), None if stream is None else _vp(int(stream)),
                                       ctypes.byref(h))
        if rc != PT_OK:
            raise PTError(rc, self.lib.pt_server_last_error(None).decode())
        self.handle = h
        self.problems = {}

    def _check(self, rc):
        if rc != PT_OK:
            raise PTError(rc, self.lib.pt_server_last_error(self.handle).decode())

    def submit(self, prob):
        keep = []
        req = _request(prob, keep)
        rid = ctypes.c_int64()
        self._check(self.lib.pt_server_submit(self.handle, ctypes.byref(req), ctypes.byref(rid)))
        self.problems[rid.value] = prob
        return rid.value

    def step(self, max_done=4096):
        ids = np.zeros(max_done, np.int64)
        n = ctypes.c_int32()
        self._check(self.lib.pt_server_step(self.handle, ids.ctypes.data_as(_p_i64), int(max_done), ctypes.byref(n)))
        return ids[: n.value].tolist()

    def result(self, rid, state=True):
        prob = self.problems[rid]
        out = np.empty((prob.R, prob.n, prob.P), np.int8) if state else None
        obs = _read_obs(prob.R, lambda o: self.lib.pt_server_read_result(
            self.handle, int(rid), None if out is None else _ptr(out), 0 if out is None else out.nbytes,
            ctypes.byref(o)), self._check)
        return out, obs

    def release(self, rid):
        self._check(self.lib.pt_server_release(self.handle, int(rid)))
        self.problems.pop(rid, None)

    def info(self):
        i = pt_server_info()
        self._check(self.lib.pt_server_get_info(self.handle, ctypes.byref(i)))
        return i

    def close(self):
        if getattr(self, "handle", None):
            self.lib.pt_server_destroy(self.handle)
            self.handle = None

    __del__ = close
