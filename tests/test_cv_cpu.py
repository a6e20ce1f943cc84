"""The oracle's cross-validated path against what it must reduce to.

* a training set equals the input module's independent row subset;
* with a weight so large that every fit stays at 0, cvl equals the count-based value of the
  definition at beta = 0 (brute-force risk sets);
* relabelling the folds changes nothing; along an L2 path, warm starts reach the cold-start fits.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import cv as ocv
from paper_2310_16238_gb300 import synth
from tests import brute
from tests.test_split_cpu import small


def test_training_set_is_the_row_subset():
    d = small(41, n=70, counting=True, valued=True)
    fold = np.random.default_rng(1).integers(0, 4, d.n)
    for k in range(4):
        a = ocv.training_set(d, fold, k)
        b = synth.subset_rows(d, np.flatnonzero(fold != k))
        for f in ("stop", "start", "event", "stratum", "col_ptr", "row_idx", "val"):
            assert np.array_equal(np.asarray(getattr(a, f)), np.asarray(getattr(b, f))), f


def test_cvl_at_zero_coefficients():
    d = small(42, n=80)
    fold = np.random.default_rng(2).integers(0, 5, d.n)
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=1e6, tol=1e-10)
    cvl, betas, infos = ocv.cv_path(d, o, fold, [1e6], n_folds=5)
    assert not np.any(betas)
    zero = np.zeros(d.p)
    ref = sum(brute.loglik(d, zero) - brute.loglik(ocv.training_set(d, fold, k), zero) for k in range(5))
    assert cvl[0] == pytest.approx(ref, rel=1e-12)


def test_fold_relabelling_changes_nothing():
    d = small(43, n=90, valued=True)
    fold = np.random.default_rng(3).integers(0, 3, d.n)
    perm = np.array([2, 0, 1])
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-12)
    a, ba, _ = ocv.cv_path(d, o, fold, [0.5, 2.0])
    b, bb, _ = ocv.cv_path(d, o, perm[fold], [0.5, 2.0])
    assert np.allclose(a, b, rtol=1e-10) and np.allclose(ba, bb, rtol=1e-10, atol=1e-12)


def test_warm_starts_reach_cold_fits():
    d = small(44, n=90, valued=True)
    fold = np.random.default_rng(4).integers(0, 3, d.n)
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-13, max_sweeps=2000)
    path = [0.1, 0.5, 2.0]
    _, betas, _ = ocv.cv_path(d, o, fold, path)
    for i, v in enumerate(path):
        cold, _ = oracle.fit(d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=v, tol=1e-13, max_sweeps=2000))
        assert np.allclose(betas[i], cold, rtol=1e-6, atol=1e-8)
