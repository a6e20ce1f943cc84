"""Time-split data sets of §2.2 and §2.3, written out row by row (oracle side).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU legs may use it; the CUDA library never does. It shares no code with
the library's device-side view and imports nothing from it.

Cut days t_1 < ... < t_C split follow-up time into the intervals I_0 = (-inf, t_1),
I_k = [t_k, t_{k+1}), I_C = [t_C, +inf). A listed covariate gets one coefficient per interval
(a step-function coefficient, §2.3), which is the same as one covariate per interval that
equals x_j on the interval and 0 elsewhere. Columns of the result: the input columns in order,
each listed column replaced by C + 1 consecutive copies (interval 0 first).

Two independent constructions of the same model:

``augment``         §2.2 literally: every subject repeated in every interval k, with
                    Y_aug = min(Y, t_{k+1}) and delta_aug = delta * 1[Y in I_k], the model
                    stratified on (stratum, interval). Right-censored data only (the paper
                    defines it for time-fixed rows); (C + 1) * N rows.
``split_counting``  counting-process rows: every row cut at the interval bounds into
                    (start, stop] pieces carrying its interval's copy of the covariates, strata
                    unchanged. Works for right-censored and counting-process input.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np


@dataclasses.dataclass
class SplitData:
    """A data set in the library's input layout (rows sorted by stratum then stop, CSC X)."""

    stop: np.ndarray
    event: np.ndarray
    col_ptr: np.ndarray
    row_idx: np.ndarray
    p: int
    start: Optional[np.ndarray] = None
    stratum: Optional[np.ndarray] = None
    val: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.stop.shape[0])

    def dense_x(self) -> np.ndarray:
        x = np.zeros((self.n, self.p))
        for j in range(self.p):
            a, b = self.col_ptr[j], self.col_ptr[j + 1]
            x[self.row_idx[a:b], j] = 1.0 if self.val is None else self.val[a:b]
        return x


def view_columns(p: int, n_cuts: int, tvc_cols: Sequence[int]):
    """First result column of every input column, and the result's column count."""
    tv = set(int(j) for j in tvc_cols)
    base, c = [], 0
    for j in range(p):
        base.append(c)
        c += n_cuts + 1 if j in tv else 1
    return base, c


def _dense_rows(data):
    """Per input row: list of (column, value) pairs."""
    rows = [[] for _ in range(data.n)]
    for j in range(data.p):
        for q in range(int(data.col_ptr[j]), int(data.col_ptr[j + 1])):
            rows[int(data.row_idx[q])].append((j, 1.0 if data.val is None else float(data.val[q])))
    return rows


def _stratum_index(data):
    """0-based rank of every row's stratum among the strata present."""
    if data.stratum is None:
        return np.zeros(data.n, np.int64)
    _, inv = np.unique(np.asarray(data.stratum), return_inverse=True)
    return inv.astype(np.int64)


def _assemble(stop, start, event, stratum, xrows, p_out, valued, source=None):
    """Sort rows by (stratum, stop, construction order) and build the CSC; with ``source``
    (the input row of every constructed row) also return it in the sorted order."""
    n = len(stop)
    order = np.lexsort((np.arange(n), np.asarray(stop), np.asarray(stratum))) if n else np.zeros(0, np.int64)
    newpos = np.empty(n, np.int64)
    newpos[order] = np.arange(n)
    cols = [[] for _ in range(p_out)]
    for i in range(n):
        for c, v in xrows[i]:
            cols[c].append((int(newpos[i]), v))
    col_ptr = np.zeros(p_out + 1, np.int64)
    ri, vv = [], []
    for c in range(p_out):
        ent = sorted(cols[c])
        col_ptr[c + 1] = col_ptr[c] + len(ent)
        ri.extend(r for r, _ in ent)
        vv.extend(v for _, v in ent)
    out = SplitData(
        stop=np.asarray(stop, np.int32)[order].copy(),
        start=None if start is None else np.asarray(start, np.int32)[order].copy(),
        event=np.asarray(event, np.uint8)[order].copy(),
        stratum=np.asarray(stratum, np.int32)[order].copy(),
        col_ptr=col_ptr, row_idx=np.asarray(ri, np.int32),
        val=np.asarray(vv, np.float64) if valued else None, p=p_out)
    if source is None:
        return out
    return out, np.asarray(source, np.int64)[order]


def augment(data, cuts: Sequence[int], tvc_cols: Sequence[int] = ()) -> SplitData:
    """The augmented data set of §2.2 (with the §2.3 covariate split), every subject in every
    interval: Y_aug = min(Y, t_{k+1}), delta_aug = delta * 1[t_k <= Y < t_{k+1}], stratum
    (s, k) with id s_index * (C + 1) + k."""
    if data.start is not None:
        raise ValueError("augment: the paper's augmentation is defined for right-censored rows")
    cuts = [int(t) for t in cuts]
    C = len(cuts)
    lo = [None] + cuts          # t_k, k = 0..C (None = -inf)
    hi = cuts + [None]          # t_{k+1} (None = +inf)
    base, p_out = view_columns(data.p, C, tvc_cols)
    tv = set(int(j) for j in tvc_cols)
    sidx = _stratum_index(data)
    xr = _dense_rows(data)
    stop, event, stratum, xrows = [], [], [], []
    for k in range(C + 1):
        for i in range(data.n):
            y = int(data.stop[i])
            in_k = (lo[k] is None or y >= lo[k]) and (hi[k] is None or y < hi[k])
            stop.append(y if hi[k] is None else min(y, hi[k]))
            event.append(1 if (data.event[i] and in_k) else 0)
            stratum.append(int(sidx[i]) * (C + 1) + k)
            xrows.append([(base[j] + (k if j in tv else 0), v) for j, v in xr[i]])
    return _assemble(stop, None, event, stratum, xrows, p_out, data.val is not None)


def split_counting(data, cuts: Sequence[int], tvc_cols: Sequence[int] = (), return_source: bool = False):
    """The same model as counting-process rows: row (start, stop] (start = before every time
    when the input has none) cut into the pieces (max(start, t_k - 1), min(stop, t_{k+1} - 1)]
    that hold at least one integer day; a piece carries the event when it ends at the row's
    stop. Strata are the input's (as 0-based indices)."""
    cuts = [int(t) for t in cuts]
    C = len(cuts)
    base, p_out = view_columns(data.p, C, tvc_cols)
    tv = set(int(j) for j in tvc_cols)
    sidx = _stratum_index(data)
    xr = _dense_rows(data)
    first = int(np.min(data.stop)) - 1 if data.n else 0
    lo_all = min(first, min(cuts) - 1)
    stop, start, event, stratum, xrows, source = [], [], [], [], [], []
    for i in range(data.n):
        a = lo_all if data.start is None else int(data.start[i])
        b = int(data.stop[i])
        for k in range(C + 1):
            pa = a if k == 0 else max(a, cuts[k - 1] - 1)
            pb = b if k == C else min(b, cuts[k] - 1)
            if not pa < pb:
                continue
            stop.append(pb)
            start.append(pa)
            event.append(1 if (data.event[i] and pb == b) else 0)
            stratum.append(int(sidx[i]))
            xrows.append([(base[j] + (k if j in tv else 0), v) for j, v in xr[i]])
            source.append(i)
    return _assemble(stop, start, event, stratum, xrows, p_out, data.val is not None,
                     source if return_source else None)
