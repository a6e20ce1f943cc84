"""The Python binding only marshals arguments (CPU: no library call is made here).

make_data / make_options / make_split turn NumPy inputs into the C structs of include/cox.h:
arrays already in the declared dtype and contiguous are passed by pointer without a copy, other
dtypes are converted once, absent optional arrays become NULL, and every scalar lands in its field.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2310_16238_gb300 import synth

cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def test_make_data_passes_arrays_by_pointer():
    d, _ = synth.stratified_sparse(n=3000, p=12, k=4)
    s, keep = cox.make_data(d)
    assert s.n_rows == d.n and s.p == d.p
    for f in ("stop", "event", "stratum", "col_ptr", "row_idx"):
        assert getattr(s, f) == getattr(d, f).ctypes.data     # no copy for the declared dtype
    assert s.start is None and s.val is None                  # NULL: no start times, binary X


def test_make_data_converts_other_dtypes_once():
    d, _ = synth.time_varying(n_subj=500, p=8, k=2, density=0.05)
    d.stop = d.stop.astype(np.int64)        # wrong width: converted, values kept
    d.row_idx = d.row_idx.astype(np.int64)
    d.val = np.linspace(0.5, 1.5, d.nnz).astype(np.float32)
    s, keep = cox.make_data(d)
    assert keep["stop"].dtype == np.int32 and np.array_equal(keep["stop"], d.stop)
    assert keep["row_idx"].dtype == np.int32 and np.array_equal(keep["row_idx"], d.row_idx)
    assert keep["val"].dtype == np.float64 and np.allclose(keep["val"], d.val)
    assert s.stop == keep["stop"].ctypes.data and s.start == d.start.ctypes.data
    assert s.val == keep["val"].ctypes.data


def test_make_options_fields():
    pen = np.array([0, 1, 1, 0], np.uint8)
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=2.5, tol=1e-7, penalize=pen)
    o.max_sweeps = 17
    s, keep = cox.make_options(o, precision=cox.COX_FP32C, tile=4096, engine=cox.COX_ENGINE_AUTO)
    assert (s.penalty, s.precision, s.lam, s.tol, s.max_sweeps, s.tile) == (cox.COX_PEN_L1, cox.COX_FP32C, 2.5, 1e-7, 17, 4096)
    assert s.penalize == pen.ctypes.data and s.stream is None
    s2, _ = cox.make_options(None)
    assert s2.penalty == cox.COX_PEN_NONE and s2.penalize is None and s2.precision == cox.COX_FP64


def test_make_split_fields():
    sp, keep = cox.make_split([10, 30], [0, 3])
    c, t = keep
    assert (sp.n_cuts, sp.n_tvc) == (2, 2) and sp.cuts == c.ctypes.data and sp.tvc_cols == t.ctypes.data
    assert list(c) == [10, 30] and list(t) == [0, 3]
    sp0, _ = cox.make_split([5])
    assert (sp0.n_cuts, sp0.n_tvc) == (1, 0) and sp0.tvc_cols is None
