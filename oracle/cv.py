"""K-fold cross-validation along a penalty path, written out plainly (oracle side).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU legs may use it; the CUDA library never does. It imports nothing from
the library.

The paper picks its L1 weight by 10-fold cross-validation (§3.2, §3.3) without naming the
criterion; this follows the cross-validated partial log-likelihood of P. Verweij and H. van
Houwelingen (Stat. Med. 12, 1993):

    cvl(v) = sum_k [ l(beta_-k(v)) - l_-k(beta_-k(v)) ]

with l the full data's log partial likelihood, l_-k that of training set k (the rows whose fold
id is not k) and beta_-k(v) the penalized fit on training set k at path value v. The path is
walked in the given order; each fit starts from its own fit at the previous value (zeros first).
"""
from __future__ import annotations

import copy
from typing import Optional, Sequence

import numpy as np

from . import fit, loglik
from .split import SplitData


def training_set(data, fold, k: int) -> SplitData:
    """The rows whose fold id is not k, in their order, with X restricted to them."""
    fold = np.asarray(fold)
    keep = np.flatnonzero(fold != k)
    new = np.full(data.n, -1, np.int64)
    new[keep] = np.arange(len(keep))
    col_ptr = np.zeros(data.p + 1, np.int64)
    rows, vals = [], []
    for j in range(data.p):
        a, b = int(data.col_ptr[j]), int(data.col_ptr[j + 1])
        for q in range(a, b):
            r = new[int(data.row_idx[q])]
            if r >= 0:
                rows.append(int(r))
                if data.val is not None:
                    vals.append(float(data.val[q]))
        col_ptr[j + 1] = len(rows)
    return SplitData(
        stop=np.asarray(data.stop)[keep].astype(np.int32), event=np.asarray(data.event)[keep].astype(np.uint8),
        start=None if data.start is None else np.asarray(data.start)[keep].astype(np.int32),
        stratum=None if data.stratum is None else np.asarray(data.stratum)[keep].astype(np.int32),
        col_ptr=col_ptr, row_idx=np.asarray(rows, np.int32),
        val=None if data.val is None else np.asarray(vals, np.float64), p=data.p)


def _with_value(opts, v):
    o = copy.copy(opts)
    if o.penalty == 1:
        o.lam = float(v)
    elif o.penalty == 2:
        o.l2_var = float(v)
    else:
        raise ValueError("the path needs an L1 or L2 penalty")
    return o


def cv_path(data, opts, fold, path: Sequence[float], n_folds: Optional[int] = None, sweeps=None):
    """cvl per path value, the full-data fits (n_path x p) and every fit's info; ``sweeps[i][m]``
    (optional) caps fit m at value i (m < K: training set m, m = K: the full data)."""
    fold = np.asarray(fold)
    K = int(n_folds) if n_folds is not None else int(fold.max()) + 1
    sets = [training_set(data, fold, k) for k in range(K)] + [data]
    prev = [None] * (K + 1)
    cvl, betas, infos = [], [], []
    for i, v in enumerate(path):
        o = _with_value(opts, v)
        cur, inf = [], []
        for m, d in enumerate(sets):
            ms = None if sweeps is None else int(sweeps[i][m])
            b, info = fit(d, o, beta0=prev[m], max_sweeps=ms)
            cur.append(b)
            inf.append(info)
        cvl.append(sum(loglik(data, cur[k]) - loglik(sets[k], cur[k]) for k in range(K)))
        betas.append(cur[K])
        infos.append(inf)
        prev = cur
    return np.array(cvl), np.array(betas), infos
