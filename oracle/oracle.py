"""ctypes binding of the plain FP64 CPU oracle (cc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
the CPU-baseline leg of bench.py.  The CUDA product path never imports it.
``build()`` compiles cc_oracle.c with gcc (-O2 -ffp-contract=off, no FMA
contraction, so that the operation order written in the source is the
order executed on x86-64 and on aarch64 alike), with OpenMP when the
compiler has it: independent rows then run on all host cores, with results
bit-identical to one thread (``threads(1)``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("eta", C.c_double),
                ("dt", C.c_double), ("kepler", C.c_int), ("max_depth", C.c_int),
                ("eta_outside", C.c_int), ("split", C.c_int), ("theta", C.c_double), ("com_max", C.c_int),
                ("pad_", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("tau_pairs", C.c_uint64), ("tau_evals", C.c_uint64),
                ("kick_pairs", C.c_uint64), ("drifts", C.c_uint64),
                ("kepler_calls", C.c_uint64), ("splits", C.c_uint64),
                ("components", C.c_uint64), ("com_pairs", C.c_uint64), ("max_depth_seen", C.c_int),
                ("pad_", C.c_int)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "pad_"}


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "cc_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC]
    r = subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True, text=True)
    if r.returncode:  # no OpenMP runtime: the serial oracle
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i64, i32p, dp = C.c_double, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double)
            P, S = C.POINTER(Params), C.POINTER(Stats)
            L.orc_tau.restype = d
            L.orc_tau.argtypes = [dp, dp, d, dp, dp, d, P, dp]
            L.orc_tau_ids.restype = d
            L.orc_tau_ids.argtypes = [i64, dp, dp, dp, P, i64, i64]
            L.orc_components.restype = i64
            L.orc_components.argtypes = [i64, dp, dp, dp, P, i32p, i64, d, i32p, S]
            L.orc_edges.restype = i64
            L.orc_edges.argtypes = [i64, dp, dp, dp, P, i32p, i64, d, i32p, i64, d, C.POINTER(C.c_int64)]
            L.orc_kick.restype = None
            L.orc_kick.argtypes = [i64, dp, dp, dp, P, i32p, i32p, i64, d, S]
            L.orc_kick_com.restype = None
            L.orc_kick_com.argtypes = [i64, dp, dp, dp, P, i32p, i32p, i64, d, S]
            L.orc_drift.restype = None
            L.orc_drift.argtypes = [i64, dp, dp, i32p, i32p, i64, d, S]
            L.orc_kepler.restype = C.c_int
            L.orc_kepler.argtypes = [i64, dp, dp, dp, d, i64, i64, d]
            L.orc_evolve_cc.restype = C.c_int
            L.orc_evolve_cc.argtypes = [i64, dp, dp, dp, P, i32p, i64, d, C.c_int, S]
            L.orc_evolve.restype = C.c_int
            L.orc_evolve.argtypes = [i64, dp, dp, dp, P, i64, S]
            L.orc_evolve_systems.restype = C.c_int
            L.orc_evolve_systems.argtypes = [i64, dp, dp, dp, P, C.POINTER(C.c_int64), i64, i64, S]
            L.orc_hold_split.restype = i64
            L.orc_hold_split.argtypes = [i64, dp, dp, dp, P, i32p, i64, d, i32p, S]
            L.orc_evolve_hold.restype = C.c_int
            L.orc_evolve_hold.argtypes = [i64, dp, dp, dp, P, i32p, i64, d, C.c_int, S]
            L.orc_evolve_ok.restype = C.c_int
            L.orc_evolve_ok.argtypes = [i64, dp, dp, dp, P, i32p, i64, i32p, i64, d, C.c_int, S]
            L.orc_set_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_energy.restype = None
            L.orc_energy.argtypes = [i64, dp, dp, dp, d, d, dp, dp, dp]
            _lib = L
        return _lib


def threads(n: int = 0) -> int:
    """Set the threads of the parallel row loops (n <= 0: unchanged);
    returns the threads they will use."""
    return int(lib().orc_set_threads(int(n)))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


SPLIT_CC, SPLIT_HOLD, SPLIT_OK = 0, 1, 2


def params(G=1.0, eps=0.0, eta=0.03, dt=1.0 / 64, kepler=False, max_depth=64, eta_outside=False, split=SPLIT_CC,
           theta=0.0, com_max=32):
    return Params(G, eps, eta, dt, int(kepler), max_depth, int(eta_outside), int(split), float(theta), int(com_max), 0)


class State:
    """A particle state (m, x3, v3) the oracle integrates in place."""

    def __init__(self, m, x3, v3):
        self.m = _f64(m).copy()
        self.x3 = _f64(x3).copy()
        self.v3 = _f64(v3).copy()
        self.n = self.m.shape[0]
        assert self.x3.shape == (3, self.n) and self.v3.shape == (3, self.n)

    def copy(self):
        return State(self.m, self.x3, self.v3)


def tau_parts(xi, vi, mi, xj, vj, mj, p: Params):
    """tau(i,j) and its parts (T_ff, dT_ff, T_fb, dT_fb, tau_ff, tau_fb)."""
    parts = np.zeros(6)
    t = lib().orc_tau(_dp(_f64(xi)), _dp(_f64(vi)), float(mi), _dp(_f64(xj)), _dp(_f64(vj)),
                      float(mj), C.byref(p), _dp(parts))
    return t, parts


def tau_ids(s: State, p: Params, i: int, j: int) -> float:
    return lib().orc_tau_ids(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), i, j)


def tau_matrix(s: State, p: Params, idx=None):
    """tau for all pairs of the given ids (diagonal +inf)."""
    idx = np.arange(s.n) if idx is None else np.asarray(idx)
    k = idx.shape[0]
    out = np.full((k, k), np.inf)
    for a in range(k):
        for b in range(a + 1, k):
            out[a, b] = out[b, a] = tau_ids(s, p, int(idx[a]), int(idx[b]))
    return out


def components(s: State, p: Params, h: float, set_ids=None, stats: Stats | None = None):
    """labels (smallest id of each member's component) and component count."""
    set_ids = np.arange(s.n, dtype=np.int32) if set_ids is None else np.ascontiguousarray(set_ids, dtype=np.int32)
    lab = np.zeros(set_ids.shape[0], dtype=np.int32)
    st = stats if stats is not None else Stats()
    k = lib().orc_components(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids),
                             set_ids.shape[0], h, _ip(lab), C.byref(st))
    if k < 0:
        raise RuntimeError(f"orc_components failed: {k}")
    return lab, int(k)


def hold_split(s: State, p: Params, h: float, set_ids=None, stats: Stats | None = None):
    """HOLD split (Sec. 2.1): labels (F's smallest id for fast members, own
    id for slow ones) and 1 if the fast set is not empty, else 0."""
    set_ids = np.arange(s.n, dtype=np.int32) if set_ids is None else np.ascontiguousarray(set_ids, dtype=np.int32)
    lab = np.zeros(set_ids.shape[0], dtype=np.int32)
    st = stats if stats is not None else Stats()
    k = lib().orc_hold_split(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids),
                             set_ids.shape[0], h, _ip(lab), C.byref(st))
    if k < 0:
        raise RuntimeError(f"orc_hold_split failed: {k}")
    return lab, int(k)


def edges(s: State, p: Params, h: float, set_ids=None, near_tol=1e-12):
    set_ids = np.arange(s.n, dtype=np.int32) if set_ids is None else np.ascontiguousarray(set_ids, dtype=np.int32)
    nn = C.c_int64(0)
    cnt = lib().orc_edges(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids), set_ids.shape[0],
                          h, None, 0, near_tol, C.byref(nn))
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    lib().orc_edges(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids), set_ids.shape[0],
                    h, _ip(out), cnt, near_tol, C.byref(nn))
    return out[:cnt], int(nn.value)


def kick(s: State, p: Params, set_ids, labels, h, stats: Stats | None = None):
    set_ids = np.ascontiguousarray(set_ids, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    st = stats if stats is not None else Stats()
    lib().orc_kick(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids), _ip(labels),
                   set_ids.shape[0], h, C.byref(st))


def kick_com(s: State, p: Params, set_ids, labels, h, stats: Stats | None = None):
    """The kick with the centre-of-mass approximation of V_CC (p.theta > 0)."""
    set_ids = np.ascontiguousarray(set_ids, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    st = stats if stats is not None else Stats()
    lib().orc_kick_com(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids), _ip(labels),
                       set_ids.shape[0], h, C.byref(st))


def drift(s: State, set_ids, labels, dt, stats: Stats | None = None):
    set_ids = np.ascontiguousarray(set_ids, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    st = stats if stats is not None else Stats()
    lib().orc_drift(s.n, _dp(s.x3), _dp(s.v3), _ip(set_ids), _ip(labels), set_ids.shape[0], dt,
                    C.byref(st))


def kepler(s: State, i: int, j: int, dt: float, G: float = 1.0):
    rc = lib().orc_kepler(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), G, i, j, dt)
    if rc:
        raise RuntimeError(f"orc_kepler failed: {rc}")


def evolve_cc(s: State, p: Params, h: float, set_ids=None, stats: Stats | None = None):
    set_ids = np.arange(s.n, dtype=np.int32) if set_ids is None else np.ascontiguousarray(set_ids, dtype=np.int32)
    st = stats if stats is not None else Stats()
    rc = lib().orc_evolve_cc(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids),
                             set_ids.shape[0], h, 0, C.byref(st))
    if rc:
        raise RuntimeError(f"orc_evolve_cc failed: {rc}")
    return st


def evolve_ok(s: State, p: Params, h: float, set_ids=None, pairs=None, stats: Stats | None = None):
    """evolve_ok(S, I, h) of the OK split (Sec. 4.2): I = every pair of the
    set when pairs is None, else an (npairs, 2) array of ids (a < b, sorted)."""
    set_ids = np.arange(s.n, dtype=np.int32) if set_ids is None else np.ascontiguousarray(set_ids, dtype=np.int32)
    st = stats if stats is not None else Stats()
    if pairs is None:
        pp, npairs = None, 0
    else:
        pa = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        pp, npairs = _ip(pa), pa.shape[0]
    rc = lib().orc_evolve_ok(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids),
                             set_ids.shape[0], pp, npairs, h, 0, C.byref(st))
    if rc:
        raise RuntimeError(f"orc_evolve_ok failed: {rc}")
    return st


def evolve_hold(s: State, p: Params, h: float, set_ids=None, stats: Stats | None = None):
    """evolve_hold(S, h) of Sec. 2.1 (Eq. HOLD) on the given set."""
    set_ids = np.arange(s.n, dtype=np.int32) if set_ids is None else np.ascontiguousarray(set_ids, dtype=np.int32)
    st = stats if stats is not None else Stats()
    rc = lib().orc_evolve_hold(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), _ip(set_ids),
                               set_ids.shape[0], h, 0, C.byref(st))
    if rc:
        raise RuntimeError(f"orc_evolve_hold failed: {rc}")
    return st


def evolve(s: State, p: Params, nsteps: int, stats: Stats | None = None, sys_off=None):
    st = stats if stats is not None else Stats()
    if sys_off is None:
        rc = lib().orc_evolve(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p), nsteps, C.byref(st))
    else:
        off = np.ascontiguousarray(sys_off, dtype=np.int64)
        rc = lib().orc_evolve_systems(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), C.byref(p),
                                      off.ctypes.data_as(C.POINTER(C.c_int64)), off.shape[0] - 1,
                                      nsteps, C.byref(st))
    if rc:
        raise RuntimeError(f"orc_evolve failed: {rc}")
    return st


def energy(s: State, G=1.0, eps=0.0):
    E = C.c_double(0.0)
    P = np.zeros(3)
    L = np.zeros(3)
    lib().orc_energy(s.n, _dp(s.x3), _dp(s.v3), _dp(s.m), G, eps, C.byref(E), _dp(P), _dp(L))
    return float(E.value), P, L
