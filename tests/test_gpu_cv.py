"""Cross-validated penalty path (cox_cv_path) on the GPU against the oracle's path.

Training sets are built on the device from the fold ids; every value's K + 1 fits run as one
batch with warm starts. The oracle walks the same path with each fit capped at the GPU fit's
sweep count (iterate-level parity): beta 1e-9 relative, cvl within 1e-9 of the scale of its
log-likelihood terms, the same best index.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import cv as ocv
from paper_2310_16238_gb300 import synth
from tests.test_gpu_split import mid

pytestmark = pytest.mark.gpu

cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if b.size else 0.0


def _check(d, o, fold, path, K, precision=None):
    kw = {} if precision is None else {"precision": precision}
    r = cox.cox_cv_path(d, fold, path, o, n_folds=K, **kw)
    sweeps = [[f["sweeps"] for f in row] for row in r["info"]]
    cvl, betas, infos = ocv.cv_path(d, o, fold, path, n_folds=K, sweeps=sweeps)
    scale = sum(abs(f["loglik"]) for row in infos for f in row)
    assert np.max(np.abs(r["cvl"] - cvl)) <= 1e-9 * scale
    for i in range(len(path)):
        assert _rel(r["beta"][i], betas[i]) <= 1e-9 or not np.any(betas[i]) and not np.any(r["beta"][i])
    assert r["best"] == int(np.argmax(cvl))
    return r


def test_cv_l1_path_stratified():
    d = mid(51, n=5000, p=10, n_strata=4)
    fold = cox.make_folds(d.n, 5, seed=1)
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=0.0, tol=1e-9)
    r = _check(d, o, fold, [40.0, 20.0, 10.0, 5.0, 2.0], 5)
    assert all(len(row) == 6 for row in r["info"])


def test_cv_l2_path_counting():
    data, o = synth.time_varying(n_subj=3000, p=8, k=3, density=0.05, event_frac=0.3, n_support=4, seed=52)
    # one fold id per row here (the generator keeps no subject id); both sides use the same folds
    fold = cox.make_folds(data.n, 4, seed=2)
    _check(data, o, fold, [0.02, 0.1, 0.5], 4)


def test_cv_valued_columns_l2():
    d = mid(53, n=3000, p=6, valued=True)
    fold = cox.make_folds(d.n, 3, seed=3)
    _check(d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9), fold, [0.05, 0.5, 5.0], 3)


def test_cv_device_folds_and_fp32c():
    import torch
    d = mid(54, n=4000, p=8)
    fold = cox.make_folds(d.n, 4, seed=4)
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=0.0, tol=1e-9)
    a = cox.cox_cv_path(d, fold, [10.0, 3.0], o, n_folds=4)
    b = cox.cox_cv_path(d, torch.from_numpy(fold).cuda(), [10.0, 3.0], o, n_folds=4)
    assert np.array_equal(a["cvl"], b["cvl"]) and np.array_equal(a["beta"], b["beta"])
    c = cox.cox_cv_path(d, fold, [10.0, 3.0], o, n_folds=4, precision=cox.COX_FP32C)
    assert np.max(np.abs(c["beta"] - a["beta"])) <= 1e-5 * max(np.max(np.abs(a["beta"])), 1e-12)


@pytest.mark.parametrize("bad", ["one_fold", "fold_range", "no_penalty", "negative_weight"])
def test_cv_rejects_bad_arguments(bad):
    d = mid(55, n=500, p=4)
    fold = cox.make_folds(d.n, 3, seed=5)
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=0.0, tol=1e-9)
    path, K = [1.0], 3
    if bad == "one_fold":
        K = 1
    elif bad == "fold_range":
        fold = fold.copy()
        fold[7] = 3
    elif bad == "no_penalty":
        o = synth.CoxOptions(penalty=synth.PEN_NONE)
    else:
        path = [-1.0]
    with pytest.raises(cox.CoxError) as e:
        cox.cox_cv_path(d, fold, path, o, n_folds=K)
    assert e.value.code == cox.COX_E_INVALID


def test_cv_on_the_time_split_view():
    """10-fold-style CV of a model whose treatment coefficient steps at a cut day (the paper's
    §3.3 workflow): training sets and the full data are split on the device; the oracle walks
    the same path on its counting-process split, each piece in its source row's fold."""
    from oracle import split as osplit
    d = mid(56, n=3000, p=8, n_strata=3)
    fold = cox.make_folds(d.n, 4, seed=6)
    cuts, tvc = [60, 140], [0, 5]
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9)
    path = [0.1, 0.5, 2.0]
    r = cox.cox_cv_path(d, fold, path, o, n_folds=4, cuts=cuts, tvc_cols=tvc)
    pv = osplit.view_columns(d.p, len(cuts), tvc)[1]
    assert r["beta"].shape == (len(path), pv)
    sc, src = osplit.split_counting(d, cuts, tvc, return_source=True)
    sweeps = [[f["sweeps"] for f in row] for row in r["info"]]
    cvl, betas, infos = ocv.cv_path(sc, o, fold[src], path, n_folds=4, sweeps=sweeps)
    scale = sum(abs(f["loglik"]) for row in infos for f in row)
    assert np.max(np.abs(r["cvl"] - cvl)) <= 1e-9 * scale
    for i in range(len(path)):
        assert _rel(r["beta"][i], betas[i]) <= 1e-9
