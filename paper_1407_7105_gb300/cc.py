"""ctypes binding of libcc.so (include/cc.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
torch tensors / numpy arrays to pointers, passes torch's current CUDA
stream, and turns negative return codes into exceptions.  Importing it
without a built libcc.so raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcc.so")

PREC_FP64 = 0
PREC_MIXED = 1
SPLIT_CC = 0
SPLIT_HOLD = 1
SPLIT_OK = 2
SMALL_AUTO = -1

ERRORS = {-1: "CC_E_ARG", -2: "CC_E_CUDA", -3: "CC_E_DEPTH", -4: "CC_E_TIMEOUT", -5: "CC_E_NONFINITE",
          -6: "CC_E_CAPACITY", -7: "CC_E_KEPLER", -8: "CC_E_NOMEM"}


class Params(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("eta", C.c_double), ("dt", C.c_double),
                ("h_fp64", C.c_double), ("near_tol", C.c_double), ("precision", C.c_int),
                ("kepler", C.c_int), ("max_depth", C.c_int), ("s_small", C.c_int),
                ("eta_outside", C.c_int), ("autotune", C.c_int), ("edge_rec_max", C.c_int),
                ("fault_test", C.c_int), ("split", C.c_int), ("com_max", C.c_int), ("theta", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("tau_pairs", C.c_uint64), ("tau_fp64", C.c_uint64), ("kick_pairs", C.c_uint64),
                ("drifts", C.c_uint64), ("kepler_calls", C.c_uint64), ("splits", C.c_uint64),
                ("components", C.c_uint64), ("edges", C.c_uint64), ("near_pairs", C.c_uint64),
                ("small_tasks", C.c_uint64), ("launches", C.c_uint64), ("tau_evaluated", C.c_uint64),
                ("com_pairs", C.c_uint64), ("max_depth_seen", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "reserved"}


class Timing(C.Structure):
    _fields_ = [("tau_ms", C.c_double), ("kick_ms", C.c_double), ("small_ms", C.c_double),
                ("tau_launches", C.c_int64), ("kick_launches", C.c_int64), ("small_launches", C.c_int64),
                ("tau_pairs", C.c_uint64), ("kick_pairs", C.c_uint64),
                ("small_tau_evaluated", C.c_uint64), ("small_kick_pairs", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneEntry(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("bin", C.c_int32), ("best", C.c_int32), ("nvar", C.c_int32),
                ("shape", C.c_int32 * 3), ("slices", C.c_int32 * 3), ("timed", C.c_int32 * 3),
                ("reserved", C.c_int32), ("us_per_mpair", C.c_double * 3)]


TUNE_KERNELS = ("tau_fp64", "tau_mixed", "kick_fp64", "kick_mixed")


class CCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None

EXPORTS = ["cc_default_params", "cc_init", "cc_set_systems", "cc_set_stream", "cc_timestep_graph",
           "cc_components", "cc_kick", "cc_drift", "cc_evolve", "cc_get_state", "cc_set_state", "cc_stats",
           "cc_reset_stats", "cc_energy", "cc_near_pairs", "cc_set_timing", "cc_timing", "cc_tuning", "cc_probe_peaks",
           "cc_components_noalloc", "cc_destroy", "cc_last_error"]


def lib():
    """Load libcc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcc.so not built ({LIB_PATH}); run paper_1407_7105_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32p, dp = C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p
        L.cc_default_params.argtypes = [C.POINTER(Params)]
        L.cc_init.argtypes = [C.POINTER(vp), i64, dp, dp, dp, C.POINTER(Params), vp]
        L.cc_set_systems.argtypes = [vp, C.POINTER(C.c_int64), i64]
        L.cc_set_stream.argtypes = [vp, vp]
        L.cc_timestep_graph.argtypes = [vp, i32p, i64, C.c_double, C.POINTER(C.c_int64), i32p, i64,
                                        C.POINTER(C.c_int64)]
        L.cc_components.argtypes = [vp, i32p, i64, C.c_double, i32p, C.POINTER(C.c_int64)]
        L.cc_kick.argtypes = [vp, i32p, i64, i32p, C.c_double]
        L.cc_drift.argtypes = [vp, i32p, i64, i32p, C.c_double]
        L.cc_evolve.argtypes = [vp, C.c_double, C.c_double]
        L.cc_get_state.argtypes = [vp, C.POINTER(C.c_double), dp, dp, dp]
        L.cc_set_state.argtypes = [vp, C.c_double, dp, dp, dp]
        L.cc_stats.argtypes = [vp, C.POINTER(Stats)]
        L.cc_reset_stats.argtypes = [vp]
        L.cc_energy.argtypes = [vp, C.POINTER(C.c_double), dp, dp]
        L.cc_near_pairs.argtypes = [vp, i32p, dp, i64, C.POINTER(C.c_int64)]
        L.cc_set_timing.argtypes = [vp, C.c_int]
        L.cc_timing.argtypes = [vp, C.POINTER(Timing)]
        L.cc_tuning.argtypes = [vp, C.POINTER(TuneEntry), i64, C.POINTER(C.c_int64)]
        L.cc_probe_peaks.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.cc_components_noalloc.argtypes = [dp, dp, dp, i64, C.POINTER(Params), C.c_double, i32p, vp, vp]
        L.cc_destroy.argtypes = [vp]
        L.cc_last_error.argtypes = [vp]
        L.cc_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name != "cc_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def default_params(**kw) -> Params:
    p = Params()
    lib().cc_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(a):
    """Pointer of a torch tensor (host or CUDA) or numpy array; None -> NULL."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    raise TypeError(type(a))


def _stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def probe_peaks(stream=None):
    """Measured FP64 and FP32 FMA throughput of the current GPU (flop/s)."""
    f64, f32 = C.c_double(0.0), C.c_double(0.0)
    rc = lib().cc_probe_peaks(stream if stream is not None else _stream(), C.byref(f64), C.byref(f32))
    if rc:
        raise CCError(rc, lib().cc_last_error(None).decode())
    return float(f64.value), float(f32.value)


def _require_cuda(name, t, dtype, numel):
    """components_noalloc's buffers are read and written by kernels: CUDA
    tensors of the stated dtype and at least `numel` elements."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def components_noalloc(m, x3, v3, h: float, labels_out, n_comp_out, params: Params | None = None, stream=None):
    """cc_components_noalloc: labels of all particles of a device-resident
    state into caller-provided device buffers (labels_out int32[n],
    n_comp_out int64[1]); the library allocates nothing."""
    import torch
    n = int(m.shape[0])
    _require_cuda("m", m, torch.float64, n)
    _require_cuda("x3", x3, torch.float64, 3 * n)
    _require_cuda("v3", v3, torch.float64, 3 * n)
    _require_cuda("labels_out", labels_out, torch.int32, n)
    _require_cuda("n_comp_out", n_comp_out, torch.int64, 1)
    p = params if params is not None else default_params()
    rc = lib().cc_components_noalloc(_ptr(m), _ptr(x3), _ptr(v3), int(m.shape[0]), C.byref(p), float(h),
                                     _ptr(labels_out), _ptr(n_comp_out),
                                     stream if stream is not None else _stream())
    if rc:
        raise CCError(rc, "cc_components_noalloc")


class Context:
    """One GPU-resident particle system driven through the C ABI."""

    def __init__(self, m, x3, v3, params: Params | None = None, stream=None, **kw):
        self._keep = (m, x3, v3)
        self.params = params if params is not None else default_params(**kw)
        n = int(m.shape[0])
        self.n = n
        h = C.c_void_p()
        rc = lib().cc_init(C.byref(h), n, _ptr(m), _ptr(x3), _ptr(v3), C.byref(self.params),
                           stream if stream is not None else _stream())
        if rc:
            raise CCError(rc, lib().cc_last_error(None).decode())
        self._h = h

    def _check(self, rc):
        if rc:
            raise CCError(rc, lib().cc_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().cc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        self._check(lib().cc_set_stream(self._h, stream if stream is not None else _stream()))

    def set_systems(self, sys_off):
        off = np.ascontiguousarray(sys_off, dtype=np.int64)
        self._check(lib().cc_set_systems(self._h, off.ctypes.data_as(C.POINTER(C.c_int64)), off.shape[0] - 1))

    def evolve(self, t_end: float, eta: float = 0.0):
        self._check(lib().cc_evolve(self._h, float(t_end), float(eta)))

    def components(self, h: float, set_ids=None, labels_out=None):
        """labels (smallest id per component) of set_ids (ascending int32), n_comp."""
        nset = self.n if set_ids is None else int(set_ids.shape[0])
        if labels_out is None:
            labels_out = np.zeros(nset, dtype=np.int32)
        nc = C.c_int64(0)
        self._check(lib().cc_components(self._h, _ptr(set_ids), nset, float(h), _ptr(labels_out), C.byref(nc)))
        return labels_out, int(nc.value)

    def timestep_graph(self, h: float, set_ids=None, cap: int | None = None):
        nset = self.n if set_ids is None else int(set_ids.shape[0])
        ne, nn = C.c_int64(0), C.c_int64(0)
        self._check(lib().cc_timestep_graph(self._h, _ptr(set_ids), nset, float(h), C.byref(ne), None, 0,
                                            C.byref(nn)))
        cap = int(ne.value) if cap is None else cap
        out = np.zeros((max(cap, 1), 2), dtype=np.int32)
        rc = lib().cc_timestep_graph(self._h, _ptr(set_ids), nset, float(h), C.byref(ne), _ptr(out), cap,
                                     C.byref(nn))
        if rc and rc != -6:
            self._check(rc)
        return out[:min(cap, int(ne.value))], int(ne.value), int(nn.value)

    def kick(self, labels, h: float, set_ids=None):
        nset = self.n if set_ids is None else int(set_ids.shape[0])
        self._check(lib().cc_kick(self._h, _ptr(set_ids), nset, _ptr(labels), float(h)))

    def drift(self, labels, h: float, set_ids=None):
        nset = self.n if set_ids is None else int(set_ids.shape[0])
        self._check(lib().cc_drift(self._h, _ptr(set_ids), nset, _ptr(labels), float(h)))

    def get_state(self, m=None, x3=None, v3=None, alloc: bool = True):
        """Copy the state into the given buffers; missing ones are new host
        numpy arrays when alloc, else skipped."""
        n = self.n
        if alloc:
            m = np.zeros(n) if m is None else m
            x3 = np.zeros((3, n)) if x3 is None else x3
            v3 = np.zeros((3, n)) if v3 is None else v3
        t = C.c_double(0.0)
        self._check(lib().cc_get_state(self._h, C.byref(t), _ptr(m), _ptr(x3), _ptr(v3)))
        return float(t.value), m, x3, v3

    def set_state(self, t: float, m=None, x3=None, v3=None):
        self._check(lib().cc_set_state(self._h, float(t), _ptr(m), _ptr(x3), _ptr(v3)))

    def stats(self) -> dict:
        s = Stats()
        self._check(lib().cc_stats(self._h, C.byref(s)))
        return s.as_dict()

    def reset_stats(self):
        self._check(lib().cc_reset_stats(self._h))

    def energy(self):
        E = C.c_double(0.0)
        P = np.zeros(3)
        L = np.zeros(3)
        self._check(lib().cc_energy(self._h, C.byref(E), _ptr(P), _ptr(L)))
        return float(E.value), P, L

    def set_timing(self, on: bool = True):
        self._check(lib().cc_set_timing(self._h, int(on)))

    def timing(self) -> dict:
        t = Timing()
        self._check(lib().cc_timing(self._h, C.byref(t)))
        return t.as_dict()

    def tuning(self) -> list:
        """The autotuner's timed cells: one dict per (kernel, size bin)."""
        n = C.c_int64(0)
        self._check(lib().cc_tuning(self._h, None, 0, C.byref(n)))
        k = int(n.value)
        buf = (TuneEntry * max(1, k))()
        self._check(lib().cc_tuning(self._h, buf, k, C.byref(n)))
        out = []
        for e in buf[:k]:
            nv = e.nvar
            out.append({"kernel": TUNE_KERNELS[e.kernel], "bin": e.bin, "best": e.best,
                        "shape": list(e.shape[:nv]), "slices": list(e.slices[:nv]), "timed": list(e.timed[:nv]),
                        "us_per_mpair": [round(x, 3) for x in e.us_per_mpair[:nv]]})
        return out

    def near_pairs(self, cap: int = 4096):
        pairs = np.zeros((cap, 2), dtype=np.int32)
        tau = np.zeros(cap)
        n = C.c_int64(0)
        self._check(lib().cc_near_pairs(self._h, _ptr(pairs), _ptr(tau), cap, C.byref(n)))
        k = min(cap, int(n.value))
        return pairs[:k], tau[:k], int(n.value)
