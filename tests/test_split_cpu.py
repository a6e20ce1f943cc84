"""The oracle's time-split constructions (§2.2, §2.3) against definitions that do not use them.

* eq. (time_coef_l) evaluated on the unsplit data with a step-function coefficient (brute
  force) equals the log-likelihood of both constructions;
* §2.2's claim: interval stratification alone (no covariate split) leaves the likelihood and
  the CCD path unchanged;
* a cut after the last time gives the later copy of a covariate no risk set (zero derivatives),
  and the fit of the other coefficients equals the unsplit fit.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import split as osplit
from paper_2310_16238_gb300 import synth
from tests import brute


def small(seed, n=60, p=4, n_strata=3, counting=False, valued=False, days=14):
    rng = np.random.default_rng(seed)
    stop = rng.integers(1, days + 1, n)
    event = (rng.random(n) < 0.6).astype(np.uint8)
    stratum = 3 * rng.integers(0, n_strata, n) + 1 if n_strata > 1 else None
    start = (stop - rng.integers(1, 8, n)) if counting else None
    rows = [np.flatnonzero(rng.random(n) < 0.5) for _ in range(p)]
    vals = [rng.normal(size=len(r)) for r in rows] if valued else None
    return synth.finalize(stop, event, stratum, start, rows, vals, p)


CUTS = [5, 9]


@pytest.mark.parametrize("seed,counting,valued,tvc", [
    (1, False, False, [1]), (2, False, True, [0, 3]), (3, True, False, [2]), (4, True, True, [0, 1, 2, 3]),
    (5, False, False, []),
])
def test_constructions_match_step_coefficient_likelihood(seed, counting, valued, tvc):
    d = small(seed, counting=counting, valued=valued)
    assert any(int(t) in CUTS for t in d.stop[d.event == 1]), "an event on a cut day checks the interval bounds"
    sc = osplit.split_counting(d, CUTS, tvc)
    pv = osplit.view_columns(d.p, len(CUTS), tvc)[1]
    assert sc.p == pv
    rng = np.random.default_rng(seed + 100)
    for _ in range(3):
        b = rng.normal(scale=0.5, size=pv)
        ref = brute.loglik_step_coef(d, b, CUTS, tvc)
        assert oracle.loglik(sc, b) == pytest.approx(ref, rel=1e-12, abs=1e-12)
        if not counting:
            au = osplit.augment(d, CUTS, tvc)
            assert au.n == (len(CUTS) + 1) * d.n
            assert oracle.loglik(au, b) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_augment_rejects_counting_rows():
    with pytest.raises(ValueError):
        osplit.augment(small(6, counting=True), CUTS, [0])


def test_interval_strata_alone_change_nothing():
    """§2.2: stratifying on the intervals (no covariate split) leaves the partial likelihood,
    and hence every coordinate step, unchanged."""
    d = small(7, n=80, valued=True)
    au = osplit.augment(d, CUTS, [])
    b = np.random.default_rng(8).normal(scale=0.4, size=d.p)
    assert oracle.loglik(au, b) == pytest.approx(oracle.loglik(d, b), rel=1e-13)
    g, h = oracle.grad_hess(d, b)
    ga, ha = oracle.grad_hess(au, b)
    assert np.allclose(ga, g, rtol=1e-12, atol=1e-12) and np.allclose(ha, h, rtol=1e-12, atol=1e-12)
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-12)
    bf, inf = oracle.fit(d, o)
    ba, ina = oracle.fit(au, o)
    assert ina["sweeps"] == inf["sweeps"]
    assert np.allclose(ba, bf, rtol=1e-10, atol=1e-12)


def test_cut_after_last_time():
    """A cut after every time: the later copy of the split covariate never meets a risk set
    (g' = g'' = 0, coefficient stays 0) and the other coefficients equal the unsplit fit."""
    d = small(9, n=70)
    cut = [int(d.stop.max()) + 1]
    for build in (osplit.augment, osplit.split_counting):
        v = build(d, cut, [2])
        b = np.random.default_rng(10).normal(scale=0.3, size=v.p)
        g, h = oracle.grad_hess(v, b)
        assert g[3] == 0.0 and h[3] == 0.0
        o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=2.0, tol=1e-12)
        bv, _ = oracle.fit(v, o)
        bp, _ = oracle.fit(d, o)
        assert bv[3] == 0.0
        assert np.allclose(np.delete(bv, 3), bp, rtol=1e-9, atol=1e-12)


def test_cut_before_first_time():
    """A cut at or before the first time: interval 0 holds no event, so the earlier copy has
    zero derivatives and the later copy carries the whole fit."""
    d = small(11, n=70)
    cut = [int(d.stop.min())]
    v = osplit.split_counting(d, cut, [1])
    b = np.zeros(v.p)
    g, h = oracle.grad_hess(v, b)
    assert g[1] == 0.0 and h[1] == 0.0
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=2.0, tol=1e-12)
    bv, _ = oracle.fit(v, o)
    bp, _ = oracle.fit(d, o)
    assert bv[1] == 0.0
    assert np.allclose(np.delete(bv, 1), bp, rtol=1e-9, atol=1e-12)
