"""ctypes binding of ``libcoxgb.so`` (C ABI in ``include/cox.h``).

Argument marshalling only: every computation runs in the library's CUDA kernels. Arrays
may be NumPy (host) or torch CUDA tensors (device); the library detects which. When torch
has CUDA, device memory is routed through torch's caching allocator. If the library is
missing or fails to load, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library (COXGB_LIBRARY: another build of it, such as the diagnostic one of build.py --trace)
LIB_PATH = os.environ.get("COXGB_LIBRARY") or os.path.join(_HERE, "_build", "libcoxgb.so")

COX_OK, COX_W_NOT_CONVERGED = 0, 1
COX_E_INVALID, COX_E_UNSORTED, COX_E_OOM, COX_E_CUDA = -1, -2, -3, -4
COX_E_TIMEOUT, COX_E_ADMISSION, COX_E_RANGE, COX_E_NOT_FOUND, COX_E_BUSY = -5, -6, -7, -8, -9
COX_PEN_NONE, COX_PEN_L1, COX_PEN_L2 = 0, 1, 2
COX_FP64, COX_FP32C = 0, 1
COX_ENGINE_AUTO, COX_ENGINE_STREAM, COX_ENGINE_RESIDENT, COX_ENGINE_INCR = 0, 1, 2, 3

EXPORTS = ["cox_set_allocator", "cox_create", "cox_set_options", "cox_fit", "cox_loglik", "cox_gradient",
           "cox_risk_sums", "cox_metadata", "cox_dx", "cox_destroy", "cox_last_error", "cox_batch_fit",
           "cox_clone", "cox_footprint", "cox_launch_count", "cox_segscan", "cox_split_columns", "cox_create_split", "cox_cv_path",
           "cox_segscan_noalloc", "cox_debug_set_wait_limit", "cox_debug_set_chunk_tiles", "cox_set_chunk_plan", "cox_debug_set_cached_s0", "cox_shard_setup", "cox_shard_head",
           "cox_shard_partial", "cox_shard_step", "cox_shard_beta", "cox_server_create", "cox_server_submit", "cox_server_poll",
           "cox_server_wait", "cox_server_cancel", "cox_server_stats_get", "cox_server_destroy"]


class CoxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class cox_data(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("p", C.c_int32), ("reserved", C.c_int32), ("stop", C.c_void_p),
                ("start", C.c_void_p), ("event", C.c_void_p), ("stratum", C.c_void_p), ("col_ptr", C.c_void_p),
                ("row_idx", C.c_void_p), ("val", C.c_void_p)]


class cox_options(C.Structure):
    _fields_ = [("penalty", C.c_int32), ("precision", C.c_int32), ("lam", C.c_double), ("l2_var", C.c_double),
                ("penalize", C.c_void_p), ("tol", C.c_double), ("max_sweeps", C.c_int32), ("tile", C.c_int32),
                ("stream", C.c_void_p), ("engine", C.c_int32), ("reserved", C.c_int32)]


class cox_fit_info(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("converged", C.c_int32), ("coord_updates", C.c_int64),
                ("loglik", C.c_double), ("objective", C.c_double), ("status", C.c_int32), ("engine", C.c_int32),
                ("step_launches", C.c_int64), ("sweep_ms", C.c_double), ("wait_ms", C.c_double),
                ("total_ms", C.c_double)]

    def as_dict(self):
        return dict(sweeps=self.sweeps, converged=bool(self.converged), coord_updates=self.coord_updates,
                    loglik=self.loglik, objective=self.objective, status=self.status,
                    engine=self.engine, step_launches=self.step_launches, sweep_ms=self.sweep_ms, wait_ms=self.wait_ms,
                    total_ms=self.total_ms)


class cox_split(C.Structure):
    _fields_ = [("n_cuts", C.c_int32), ("n_tvc", C.c_int32), ("cuts", C.c_void_p), ("tvc_cols", C.c_void_p)]


class cox_cv(C.Structure):
    _fields_ = [("n_folds", C.c_int32), ("n_path", C.c_int32), ("fold", C.c_void_p), ("path", C.c_void_p),
                ("split", C.c_void_p)]


class cox_server_options(C.Structure):
    _fields_ = [("memory_budget", C.c_size_t), ("max_active", C.c_int32), ("precision", C.c_int32),
                ("steps_per_replay", C.c_int32), ("reserved", C.c_int32)]


class cox_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("queued", C.c_int32),
                ("preparing", C.c_int32), ("running", C.c_int32), ("done_unpolled", C.c_int32),
                ("bytes_in_use", C.c_size_t), ("memory_budget", C.c_size_t), ("replays", C.c_int64),
                ("step_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)
_lock = threading.Lock()
_lib = None
_cb_keep = []


def lib():
    """Load the library (raises if it has not been built or cannot be loaded)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            L.cox_set_allocator.argtypes = [_ALLOC, _FREE, vp]
            L.cox_create.argtypes = [C.POINTER(cox_data), C.POINTER(cox_options), C.POINTER(vp)]
            L.cox_set_options.argtypes = [vp, C.POINTER(cox_options)]
            L.cox_fit.argtypes = [vp, vp, vp, C.POINTER(cox_fit_info)]
            L.cox_loglik.argtypes = [vp, vp, vp]
            L.cox_gradient.argtypes = [vp, vp, vp, vp]
            L.cox_risk_sums.argtypes = [vp, vp, i32, vp, vp, vp]
            L.cox_metadata.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            L.cox_dx.argtypes = [vp, vp]
            L.cox_destroy.argtypes = [vp]
            L.cox_destroy.restype = None
            L.cox_last_error.argtypes = [vp]
            L.cox_last_error.restype = C.c_char_p
            L.cox_batch_fit.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(cox_fit_info)]
            L.cox_clone.argtypes = [vp, C.POINTER(cox_options), C.POINTER(vp)]
            L.cox_footprint.argtypes = [C.POINTER(cox_data), C.POINTER(cox_options), C.POINTER(C.c_size_t)]
            L.cox_split_columns.argtypes = [i32, C.POINTER(cox_split), C.POINTER(i32)]
            L.cox_create_split.argtypes = [C.POINTER(cox_data), C.POINTER(cox_split), C.POINTER(cox_options), C.POINTER(vp)]
            L.cox_cv_path.argtypes = [C.POINTER(cox_data), C.POINTER(cox_options), C.POINTER(cox_cv), vp, vp,
                                      C.POINTER(cox_fit_info), C.POINTER(i32)]
            L.cox_launch_count.argtypes = []
            L.cox_launch_count.restype = i64
            L.cox_segscan.argtypes = [vp, vp, i64, vp, vp]
            L.cox_segscan_noalloc.argtypes = [vp, vp, i64, vp, vp]
            L.cox_debug_set_wait_limit.argtypes = [C.c_longlong]
            L.cox_debug_set_chunk_tiles.argtypes = [C.c_int32]
            L.cox_set_chunk_plan.argtypes = [C.c_int32]
            L.cox_debug_set_cached_s0.argtypes = [C.c_int32]
            L.cox_shard_setup.argtypes = [vp, vp, i32]
            L.cox_shard_head.argtypes = [vp, i32, vp]
            L.cox_shard_partial.argtypes = [vp, i32, vp, i32, vp]
            L.cox_shard_step.argtypes = [vp, i32, vp, i32, i32, i32, C.POINTER(i32), C.POINTER(C.c_double)]
            L.cox_shard_beta.argtypes = [vp, vp]
            L.cox_server_create.argtypes = [C.POINTER(cox_server_options), C.POINTER(vp)]
            L.cox_server_submit.argtypes = [vp, C.POINTER(cox_data), C.POINTER(cox_options), C.POINTER(C.c_uint64)]
            L.cox_server_poll.argtypes = [vp, C.c_uint64, vp, C.POINTER(cox_fit_info)]
            L.cox_server_wait.argtypes = [vp, C.c_uint64, C.c_double, vp, C.POINTER(cox_fit_info)]
            L.cox_server_cancel.argtypes = [vp, C.c_uint64]
            L.cox_server_stats_get.argtypes = [vp, C.POINTER(cox_server_stats)]
            L.cox_server_destroy.argtypes = [vp]
            L.cox_server_destroy.restype = None
            _lib = L
            _install_torch_allocator(L)
    return _lib


def _install_torch_allocator(L):
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except Exception:
        return

    def alloc(nbytes, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:
            return None

    def free(ptr, nbytes, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC(alloc), _FREE(free)
    _cb_keep.extend([a, f])
    L.cox_set_allocator(a, f, None)


def _check(rc, handle=None, allow_warn=True):
    if rc < 0 or (rc > 0 and not allow_warn):
        msg = lib().cox_last_error(handle).decode()
        raise CoxError(rc, msg)
    return rc


def _ptr(a):
    """Pointer of a NumPy array or torch tensor (None stays None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def make_data(data):
    """cox_data for a ``synth.CoxData`` or any object with the same fields (NumPy or torch)."""
    def conv(x, dt):
        if x is None:
            return None
        if hasattr(x, "data_ptr"):
            return x.contiguous()
        return _host(x, dt)
    keep = dict(stop=conv(data.stop, np.int32), start=conv(data.start, np.int32), event=conv(data.event, np.uint8),
                stratum=conv(data.stratum, np.int32), col_ptr=conv(data.col_ptr, np.int64),
                row_idx=conv(data.row_idx, np.int32), val=conv(data.val, np.float64))
    n = int(keep["stop"].shape[0])
    d = cox_data(n, int(data.p), 0, _ptr(keep["stop"]), _ptr(keep["start"]), _ptr(keep["event"]),
                 _ptr(keep["stratum"]), _ptr(keep["col_ptr"]), _ptr(keep["row_idx"]), _ptr(keep["val"]))
    return d, keep


def make_options(opts=None, precision=COX_FP64, stream=None, tile=0, engine=COX_ENGINE_AUTO):
    """cox_options from a ``synth.CoxOptions``-like object."""
    pen = None
    if opts is not None and getattr(opts, "penalize", None) is not None:
        pen = _host(opts.penalize, np.uint8)
    o = cox_options(int(getattr(opts, "penalty", COX_PEN_NONE)), int(precision), float(getattr(opts, "lam", 0.0)),
                    float(getattr(opts, "l2_var", 1.0)), _ptr(pen), float(getattr(opts, "tol", 1e-8)),
                    int(getattr(opts, "max_sweeps", 1000)), int(tile), stream, int(engine), 0)
    return o, pen


# ---------------------------------------------------------------- ABI-named wrappers
def cox_create(data, opts=None, precision=COX_FP64, stream=None, tile=0, engine=COX_ENGINE_AUTO):
    d, keep = make_data(data)
    o, pen = make_options(opts, precision, stream, tile, engine)
    h = C.c_void_p()
    _check(lib().cox_create(C.byref(d), C.byref(o), C.byref(h)))
    _P_CACHE[h.value] = int(data.p)
    return h


def make_split(cuts, tvc_cols=()):
    """cox_split for cut days ``cuts`` (ascending) and the columns ``tvc_cols`` that get one
    coefficient per interval."""
    c = np.ascontiguousarray(cuts, dtype=np.int32)
    t = np.ascontiguousarray(tvc_cols, dtype=np.int32)
    sp = cox_split(int(c.shape[0]), int(t.shape[0]), _ptr(c), _ptr(t) if t.shape[0] else None)
    return sp, (c, t)


def cox_split_columns(p, cuts, tvc_cols=()):
    sp, keep = make_split(cuts, tvc_cols)
    out = C.c_int32()
    _check(lib().cox_split_columns(int(p), C.byref(sp), C.byref(out)))
    return int(out.value)


def cox_create_split(data, cuts, tvc_cols=(), opts=None, precision=COX_FP64, stream=None, tile=0,
                     engine=COX_ENGINE_AUTO):
    """Handle on the time-split view of ``data`` (§2.2, §2.3); its p is the view's."""
    d, keep = make_data(data)
    sp, skeep = make_split(cuts, tvc_cols)
    o, pen = make_options(opts, precision, stream, tile, engine)
    h = C.c_void_p()
    _check(lib().cox_create_split(C.byref(d), C.byref(sp), C.byref(o), C.byref(h)))
    _P_CACHE[h.value] = cox_split_columns(data.p, cuts, tvc_cols)
    return h


def cox_cv_path(data, folds, path, opts, n_folds=None, precision=COX_FP64, stream=None, engine=COX_ENGINE_AUTO,
                cuts=None, tvc_cols=()):
    """Cross-validated penalty path (cox_cv_path): ``folds`` holds a fold id per row, ``path``
    the L1 weights (or L2 variances) in the order to walk. Returns a dict with ``cvl`` (per path
    value), ``beta`` (n_path x p full-data fits), ``best`` (index of the largest cvl) and
    ``info`` (per value: the training fits, then the full-data fit). With ``cuts`` every fit is
    on the time-split view (cox_create_split) and ``beta`` has the view's columns."""
    d, keep = make_data(data)
    sp, skeep = (None, None) if cuts is None else make_split(cuts, tvc_cols)
    o, pen = make_options(opts, precision, stream, 0, engine)
    f = folds.contiguous() if hasattr(folds, "data_ptr") else np.ascontiguousarray(folds, dtype=np.int32)
    K = int(n_folds) if n_folds is not None else int((f.max().item() if hasattr(f, "data_ptr") else f.max()) + 1)
    pth = np.ascontiguousarray(path, dtype=np.float64)
    L = int(pth.shape[0])
    cv = cox_cv(K, L, _ptr(f), _ptr(pth), C.cast(C.pointer(sp), C.c_void_p) if sp is not None else None)
    p_out = int(data.p) if cuts is None else cox_split_columns(data.p, cuts, tvc_cols)
    cvl = np.zeros(L)
    beta = np.zeros((L, max(p_out, 1)))
    infos = (cox_fit_info * (L * (K + 1)))()
    best = C.c_int32(-1)
    rc = _check(lib().cox_cv_path(C.byref(d), C.byref(o), C.byref(cv), _ptr(cvl), _ptr(beta), infos, C.byref(best)))
    info = [[infos[i * (K + 1) + m].as_dict() for m in range(K + 1)] for i in range(L)]
    return dict(cvl=cvl, beta=beta[:, :p_out], best=int(best.value), info=info, status=rc)


def make_folds(n_rows, n_folds, seed=0, subject=None):
    """Fold id per row: subjects (``subject[r]``, default one per row) dealt to the folds in a
    seeded random order, so the folds differ in size by at most one subject."""
    rng = np.random.default_rng(seed)
    subj = np.arange(n_rows) if subject is None else np.asarray(subject)
    uniq, inv = np.unique(subj, return_inverse=True)
    order = rng.permutation(len(uniq))
    fold_of = np.empty(len(uniq), np.int32)
    fold_of[order] = np.arange(len(uniq)) % n_folds
    return fold_of[inv].astype(np.int32)


def cox_fit(h, beta0=None, out=None):
    p = _num_cols(h)
    beta = np.zeros(p) if out is None else out
    b0 = None if beta0 is None else (beta0 if hasattr(beta0, "data_ptr") else _host(beta0, np.float64))
    info = cox_fit_info()
    rc = _check(lib().cox_fit(h, _ptr(b0), _ptr(beta), C.byref(info)), h)
    return beta, dict(info.as_dict(), rc=rc)


def cox_loglik(h, beta):
    b = beta if hasattr(beta, "data_ptr") else _host(beta, np.float64)
    out = np.zeros(1)
    _check(lib().cox_loglik(h, _ptr(b), _ptr(out)), h)
    return float(out[0])


def cox_gradient(h, beta, hessian=True):
    p = _num_cols(h)
    b = beta if hasattr(beta, "data_ptr") else _host(beta, np.float64)
    g = np.zeros(max(p, 1))
    hd = np.zeros(max(p, 1)) if hessian else None
    _check(lib().cox_gradient(h, _ptr(b), _ptr(g), _ptr(hd)), h)
    return (g[:p], hd[:p]) if hessian else g[:p]


def cox_risk_sums(h, beta, j):
    G = C.c_int64()
    _check(lib().cox_risk_sums(h, None, int(j), None, None, C.byref(G)), h)
    n = G.value
    s0, s1 = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    b = None if beta is None else (beta if hasattr(beta, "data_ptr") else _host(beta, np.float64))
    _check(lib().cox_risk_sums(h, _ptr(b), int(j), _ptr(s0), _ptr(s1), None), h)
    return s0[:n], s1[:n]


def cox_metadata(h):
    G, K = C.c_int64(), C.c_int64()
    _check(lib().cox_metadata(h, C.byref(G), C.byref(K), None, None, None, None, None), h)
    g, k = G.value, K.value
    gs, gt, ge = (np.zeros(max(g, 1), np.int32) for _ in range(3))
    ga = np.zeros(max(g, 1), np.int64)
    ss = np.zeros(k + 1, np.int64)
    _check(lib().cox_metadata(h, None, None, _ptr(gs), _ptr(gt), _ptr(ge), _ptr(ga), _ptr(ss)), h)
    return dict(group_stratum=gs[:g], group_time=gt[:g], group_events=ge[:g], group_at_risk=ga[:g], strata_start=ss)


def cox_dx(h):
    p = _num_cols(h)
    out = np.zeros(max(p, 1))
    _check(lib().cox_dx(h, _ptr(out)), h)
    return out[:p]


def cox_set_options(h, opts=None, precision=COX_FP64, stream=None, tile=0):
    o, pen = make_options(opts, precision, stream, tile)
    _check(lib().cox_set_options(h, C.byref(o)), h)


def cox_clone(h, opts=None, precision=COX_FP64, stream=None):
    o, pen = make_options(opts, precision, stream)
    out = C.c_void_p()
    _check(lib().cox_clone(h, C.byref(o), C.byref(out)))
    _P_CACHE[out.value] = _P_CACHE.get(h.value if isinstance(h, C.c_void_p) else h)
    return out


def cox_destroy(h):
    if h:
        _P_CACHE.pop(h.value if isinstance(h, C.c_void_p) else h, None)
        lib().cox_destroy(h)


def cox_batch_fit(handles: Sequence, beta0: Optional[Sequence] = None):
    n = len(handles)
    hs = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    outs = [np.zeros(max(_num_cols(h), 1)) for h in handles]
    b0s = None
    keep = []
    if beta0 is not None:
        arr = []
        for b in beta0:
            if b is None:
                arr.append(None)
            else:
                bb = b if hasattr(b, "data_ptr") else _host(b, np.float64)
                keep.append(bb)
                arr.append(_ptr(bb))
        b0s = (C.c_void_p * n)(*arr)
    outp = (C.c_void_p * n)(*[o.ctypes.data for o in outs])
    infos = (cox_fit_info * n)()
    rc = lib().cox_batch_fit(hs, n, b0s, outp, infos)
    _check(rc)
    return [o[:_num_cols(h)] for o, h in zip(outs, handles)], [i.as_dict() for i in infos]


def cox_footprint(data, opts=None, precision=COX_FP64):
    d, keep = make_data(data)
    o, pen = make_options(opts, precision)
    out = C.c_size_t()
    _check(lib().cox_footprint(C.byref(d), C.byref(o), C.byref(out)))
    return int(out.value)


_P_CACHE = {}


def cox_launch_count() -> int:
    return int(lib().cox_launch_count())


def cox_debug_set_wait_limit(clocks: int) -> None:
    """Bound, in SM clocks, of every device-side wait of kernels launched afterwards (<= 0: the
    default). For tests of the failure path: too short a bound makes calls return COX_E_TIMEOUT."""
    _check(lib().cox_debug_set_wait_limit(int(clocks)))


def cox_debug_set_chunk_tiles(tiles: int) -> None:
    """Tiles per chunk of the FP32C streaming kernel for work lists built afterwards (0: the
    library's choice). For tests of multi-tile chunks on small data."""
    _check(lib().cox_debug_set_chunk_tiles(int(tiles)))


def cox_set_chunk_plan(chunks_per_cta: int) -> None:
    """Chunks per resident CTA in the FP32C streaming kernel's plans for work lists built
    afterwards (0: the library's default; 1..8)."""
    _check(lib().cox_set_chunk_plan(int(chunks_per_cta)))


def cox_debug_set_cached_s0(enable: bool) -> None:
    """Turn the FP32C streaming kernel's cached-S0 path on or off for work lists built afterwards
    (on by default). For tests that compare it with the full pass."""
    _check(lib().cox_debug_set_cached_s0(1 if enable else 0))


def cox_segscan(a, head_flags, out=None, stream=None):
    """Segmented inclusive scan (§2.6) of torch CUDA tensors a (float64) and head_flags (uint8)."""
    import torch
    if out is None:
        out = torch.empty_like(a)
    _check(lib().cox_segscan(a.data_ptr(), head_flags.data_ptr(), int(a.numel()), out.data_ptr(), stream))
    return out


def _num_cols(h):
    key = h.value if isinstance(h, C.c_void_p) else h
    p = _P_CACHE.get(key)
    if p is None:
        raise RuntimeError("unknown handle: create it through cox_create / Handle")
    return p


class Handle:
    """Owning wrapper: ``Handle(data, opts, precision=COX_FP64)`` then ``fit()``, ``loglik(beta)``..."""

    def __init__(self, data, opts=None, precision=COX_FP64, stream=None, tile=0, engine=COX_ENGINE_AUTO, _raw=None):
        if _raw is None:
            d, self._keep = make_data(data)
            o, self._pen = make_options(opts, precision, stream, tile, engine)
            h = C.c_void_p()
            _check(lib().cox_create(C.byref(d), C.byref(o), C.byref(h)))
            self.h = h
            self.p = int(data.p)
        else:
            self.h, self.p = _raw
        _P_CACHE[self.h.value] = self.p
        self.precision = precision

    @classmethod
    def split(cls, data, cuts, tvc_cols=(), opts=None, precision=COX_FP64, stream=None, tile=0,
              engine=COX_ENGINE_AUTO):
        """Handle on the time-split view of ``data``: cut days ``cuts``, one coefficient per
        interval for the columns ``tvc_cols`` (cox_create_split)."""
        h = cox_create_split(data, cuts, tvc_cols, opts, precision, stream, tile, engine)
        return cls(None, _raw=(h, _P_CACHE[h.value]), precision=precision)

    def fit(self, beta0=None):
        return cox_fit(self.h, beta0)

    def loglik(self, beta):
        return cox_loglik(self.h, beta)

    def gradient(self, beta, hessian=True):
        return cox_gradient(self.h, beta, hessian)

    def risk_sums(self, beta, j):
        return cox_risk_sums(self.h, beta, j)

    def metadata(self):
        return cox_metadata(self.h)

    def dx(self):
        return cox_dx(self.h)

    def set_options(self, opts, stream=None, tile=0):
        cox_set_options(self.h, opts, self.precision, stream, tile)

    def clone(self, opts=None):
        o, pen = make_options(opts, self.precision)
        out = C.c_void_p()
        _check(lib().cox_clone(self.h, C.byref(o), C.byref(out)))
        c = Handle(None, _raw=(out, self.p), precision=self.precision)
        c._pen = pen
        return c

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _P_CACHE.pop(self.h.value, None)
            lib().cox_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def batch_fit(handles: Sequence[Handle], beta0=None):
    return cox_batch_fit([h.h for h in handles], beta0)


class Server:
    """Continuous-batching fit server (cox_server_*): submit from any thread, poll or wait."""

    def __init__(self, memory_budget=0, max_active=0, precision=COX_FP64, steps_per_replay=0):
        o = cox_server_options(int(memory_budget), int(max_active), int(precision), int(steps_per_replay), 0)
        h = C.c_void_p()
        _check(lib().cox_server_create(C.byref(o), C.byref(h)))
        self.h = h
        self.precision = precision
        self._p = {}

    def submit(self, data, opts=None) -> int:
        d, keep = make_data(data)
        o, pen = make_options(opts, self.precision)
        rid = C.c_uint64()
        _check(lib().cox_server_submit(self.h, C.byref(d), C.byref(o), C.byref(rid)))
        self._p[rid.value] = int(data.p)
        return rid.value

    def _result(self, fn, rid, *args):
        p = self._p.get(rid, 0)
        beta = np.zeros(max(p, 1))
        info = cox_fit_info()
        rc = fn(self.h, C.c_uint64(rid), *args, beta.ctypes.data, C.byref(info))
        if rc == COX_E_BUSY:
            return None
        self._p.pop(rid, None)
        _check(rc)
        return beta[:p], dict(info.as_dict(), rc=rc)

    def poll(self, rid):
        """(beta, info) when the request is finished, else None."""
        return self._result(lib().cox_server_poll, rid)

    def wait(self, rid, timeout_s=-1.0):
        return self._result(lib().cox_server_wait, rid, C.c_double(timeout_s))

    def cancel(self, rid):
        _check(lib().cox_server_cancel(self.h, C.c_uint64(rid)))

    def stats(self):
        st = cox_server_stats()
        _check(lib().cox_server_stats_get(self.h, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().cox_server_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
