"""FP64 CPU oracle for the regularized stratified / time-varying Cox CCD fit (arXiv 2310.16238).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.
It shares no code with the CUDA library (``paper_2310_16238_gb300``) and imports nothing from it.

The arithmetic lives in ``cox_oracle.c`` (plain C, FP64, compensated sums); this module
compiles it with the system C compiler on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cox_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcoxoracle.so")
_lock = threading.Lock()
_lib = None

PEN_NONE, PEN_L1, PEN_L2 = 0, 1, 2


class _Data(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int32), ("stop", C.c_void_p), ("start", C.c_void_p),
                ("event", C.c_void_p), ("stratum", C.c_void_p), ("col_ptr", C.c_void_p),
                ("row_idx", C.c_void_p), ("val", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("penalty", C.c_int32), ("lam", C.c_double), ("l2_var", C.c_double),
                ("penalize", C.c_void_p), ("tol", C.c_double), ("max_sweeps", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("coord_updates", C.c_int64), ("loglik", C.c_double),
                ("objective", C.c_double), ("converged", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libcoxoracle.so`` (plain C, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cc = os.environ.get("CC", "gcc")
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([cc, "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            L.ocx_validate.argtypes = [C.POINTER(_Data)]
            L.ocx_strata.argtypes = [C.POINTER(_Data), vp]
            L.ocx_strata.restype = i64
            L.ocx_tie_groups.argtypes = [C.POINTER(_Data), vp, vp, vp, vp]
            L.ocx_tie_groups.restype = i64
            L.ocx_num_groups.argtypes = [C.POINTER(_Data)]
            L.ocx_num_groups.restype = i64
            L.ocx_risk_count.argtypes = [C.POINTER(_Data), i64, vp, vp, vp]
            L.ocx_dX.argtypes = [C.POINTER(_Data), vp]
            L.ocx_eta.argtypes = [C.POINTER(_Data), vp, vp]
            L.ocx_segscan.argtypes = [i64, vp, vp, vp]
            L.ocx_risk_sums.argtypes = [C.POINTER(_Data), vp, i32, vp, vp, vp]
            L.ocx_grad_hess.argtypes = [C.POINTER(_Data), vp, i32, vp, vp, vp]
            L.ocx_loglik.argtypes = [C.POINTER(_Data), vp, vp]
            L.ocx_step.argtypes = [dbl, dbl, dbl, vp, i32, dbl, dbl, i32]
            L.ocx_step.restype = dbl
            L.ocx_fit.argtypes = [C.POINTER(_Data), C.POINTER(_Opts), vp, vp, C.POINTER(_Info)]
            L.ocx_time_sample.argtypes = [C.POINTER(_Data), C.POINTER(_Opts), i32, vp, vp]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Bound:
    """ctypes view of a CoxData (keeps the contiguous arrays alive)."""

    def __init__(self, data):
        self.keep = dict(
            stop=np.ascontiguousarray(data.stop, dtype=np.int32),
            start=None if data.start is None else np.ascontiguousarray(data.start, dtype=np.int32),
            event=np.ascontiguousarray(data.event, dtype=np.uint8),
            stratum=None if data.stratum is None else np.ascontiguousarray(data.stratum, dtype=np.int32),
            col_ptr=np.ascontiguousarray(data.col_ptr, dtype=np.int64),
            row_idx=np.ascontiguousarray(data.row_idx, dtype=np.int32),
            val=None if data.val is None else np.ascontiguousarray(data.val, dtype=np.float64))
        k = self.keep
        self.n, self.p = int(k["stop"].shape[0]), int(data.p)
        self.s = _Data(self.n, self.p, _ptr(k["stop"]), _ptr(k["start"]), _ptr(k["event"]),
                       _ptr(k["stratum"]), _ptr(k["col_ptr"]), _ptr(k["row_idx"]), _ptr(k["val"]))


def _opts(opts, p):
    pen = None if getattr(opts, "penalize", None) is None else np.ascontiguousarray(opts.penalize, dtype=np.uint8)
    o = _Opts(int(opts.penalty), float(opts.lam), float(opts.l2_var), _ptr(pen), float(opts.tol), int(opts.max_sweeps))
    return o, pen


def validate(data) -> int:
    b = _Bound(data)
    return int(lib().ocx_validate(C.byref(b.s)))


def strata(data) -> np.ndarray:
    b = _Bound(data)
    out = np.zeros(b.n + 1, dtype=np.int64)
    K = lib().ocx_strata(C.byref(b.s), _ptr(out))
    return out[:K + 1].copy()


def tie_groups(data):
    """(head, d, t, k): first row, event count, time and stratum id of every tie group."""
    b = _Bound(data)
    n = max(b.n, 1)
    head = np.zeros(n, np.int64); d = np.zeros(n, np.int32); t = np.zeros(n, np.int32); k = np.zeros(n, np.int32)
    G = lib().ocx_tie_groups(C.byref(b.s), _ptr(head), _ptr(d), _ptr(t), _ptr(k))
    return head[:G].copy(), d[:G].copy(), t[:G].copy(), k[:G].copy()


def risk_count(data) -> np.ndarray:
    """Rows at risk at each tie group, by the definition of the risk set (O(n G): small data)."""
    b = _Bound(data)
    _, _, t, k = tie_groups(data)
    out = np.zeros(len(t), np.int64)
    lib().ocx_risk_count(C.byref(b.s), len(t), _ptr(t), _ptr(k), _ptr(out))
    return out


def dX(data) -> np.ndarray:
    b = _Bound(data)
    out = np.zeros(max(b.p, 1))
    lib().ocx_dX(C.byref(b.s), _ptr(out))
    return out[:b.p].copy()


def eta(data, beta) -> np.ndarray:
    b = _Bound(data)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    out = np.zeros(max(b.n, 1))
    lib().ocx_eta(C.byref(b.s), _ptr(beta), _ptr(out))
    return out[:b.n].copy()


def segscan(a, f) -> np.ndarray:
    """Paper §2.6 segmented inclusive scan with head flags (flag-value operator)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.uint8)
    out = np.zeros(max(len(a), 1))
    lib().ocx_segscan(len(a), _ptr(a), _ptr(f), _ptr(out))
    return out[:len(a)].copy()


def risk_sums(data, beta, j: int):
    """(S0, S1, S2) at every tie group for column j (j < 0: only S0) at coefficients beta."""
    b = _Bound(data)
    et = eta(data, beta)
    G = int(lib().ocx_num_groups(C.byref(b.s)))
    S = [np.zeros(max(G, 1)) for _ in range(3)]
    rc = lib().ocx_risk_sums(C.byref(b.s), _ptr(et), int(j), _ptr(S[0]), _ptr(S[1]), _ptr(S[2]))
    if rc:
        raise RuntimeError(f"ocx_risk_sums failed: {rc}")
    return tuple(s[:G].copy() for s in S)


def grad_hess(data, beta, cols=None):
    """Unpenalized g'(beta_j), g''(beta_j) of -loglik (eqs. strat_g, strat_h) for ``cols``."""
    b = _Bound(data)
    et = eta(data, beta)
    cols = np.arange(b.p, dtype=np.int32) if cols is None else np.ascontiguousarray(cols, dtype=np.int32)
    g1 = np.zeros(max(len(cols), 1)); g2 = np.zeros(max(len(cols), 1))
    rc = lib().ocx_grad_hess(C.byref(b.s), _ptr(et), len(cols), _ptr(cols), _ptr(g1), _ptr(g2))
    if rc:
        raise RuntimeError(f"ocx_grad_hess failed: {rc}")
    return g1[:len(cols)].copy(), g2[:len(cols)].copy()


def loglik(data, beta) -> float:
    b = _Bound(data)
    et = eta(data, beta)
    out = np.zeros(1)
    rc = lib().ocx_loglik(C.byref(b.s), _ptr(et), _ptr(out))
    if rc:
        raise RuntimeError(f"ocx_loglik failed: {rc}")
    return float(out[0])


def step(g1, g2, beta_j, tr, penalty, lam=0.0, l2_var=1.0, penalized=1):
    """One coordinate step (§2.4). Returns (applied step, new trust half-width)."""
    t = np.array([tr], dtype=np.float64)
    s = lib().ocx_step(float(g1), float(g2), float(beta_j), _ptr(t), int(penalty), float(lam), float(l2_var), int(penalized))
    return float(s), float(t[0])


def fit(data, opts, beta0=None, max_sweeps=None):
    """CCD fit (§2.4). Returns (beta, info dict)."""
    b = _Bound(data)
    o, keep = _opts(opts, b.p)
    if max_sweeps is not None:
        o.max_sweeps = int(max_sweeps)
    beta = np.zeros(max(b.p, 1))
    b0 = None if beta0 is None else np.ascontiguousarray(beta0, dtype=np.float64)
    info = _Info()
    rc = lib().ocx_fit(C.byref(b.s), C.byref(o), _ptr(b0), _ptr(beta), C.byref(info))
    if rc < 0:
        raise RuntimeError(f"ocx_fit failed: {rc}")
    return beta[:b.p].copy(), dict(sweeps=info.sweeps, coord_updates=info.coord_updates, loglik=info.loglik,
                                   objective=info.objective, converged=bool(info.converged))


def time_sample(data, opts, ncoords: int, return_beta: bool = False):
    """Run ``ncoords`` coordinate steps from beta = 0 (a bounded timing sample: the first
    ``ncoords`` steps of the fit, cyclic order). Returns a checksum, or (checksum, beta) with
    ``return_beta``."""
    b = _Bound(data)
    o, keep = _opts(opts, b.p)
    out = np.zeros(1)
    beta = np.zeros(max(b.p, 1)) if return_beta else None
    rc = lib().ocx_time_sample(C.byref(b.s), C.byref(o), int(ncoords), _ptr(out), _ptr(beta))
    if rc:
        raise RuntimeError(f"ocx_time_sample failed: {rc}")
    return (float(out[0]), beta[:b.p].copy()) if return_beta else float(out[0])
