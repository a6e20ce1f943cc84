"""Time-split view (cox_create_split, §2.2/§2.3) on the GPU against the oracle's row-by-row
constructions.

The device view (rows that can be at risk in an interval, built by kernels from the unsplit
arrays) and the oracle's data sets (the paper's full augmentation; counting-process pieces)
hold different rows but the same partial likelihood, so the CCD paths agree: beta 1e-9
relative and log-likelihood 1e-11 relative (FP64), the FP32C bounds for FP32C.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import split as osplit
from paper_2310_16238_gb300 import synth
from tests import brute
from tests.test_split_cpu import small

pytestmark = pytest.mark.gpu

cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if len(b) else 0.0


def mid(seed, n=4000, p=12, n_strata=5, counting=False, valued=False, days=200):
    """A few thousand rows: several tiles of every engine, ragged strata."""
    rng = np.random.default_rng(seed)
    stop = rng.integers(1, days + 1, n)
    event = (rng.random(n) < 0.3).astype(np.uint8)
    stratum = rng.integers(0, n_strata, n) if n_strata > 1 else None
    start = (stop - rng.integers(1, 60, n)) if counting else None
    dens = np.exp(rng.uniform(np.log(0.01), np.log(0.4), p))
    rows = [np.flatnonzero(rng.random(n) < dd) for dd in dens]
    vals = [rng.normal(size=len(r)) for r in rows] if valued else None
    return synth.finalize(stop, event, stratum, start, rows, vals, p)


CASES = [
    ("small_rc_l2", lambda: small(21), [5, 9], [1], synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-10)),
    ("small_cp_l1", lambda: small(22, counting=True), [4, 8, 11], [0, 2],
     synth.CoxOptions(penalty=synth.PEN_L1, lam=0.5, tol=1e-10)),
    ("mid_rc_l1", lambda: mid(23), [30, 100], [0, 5, 11], synth.CoxOptions(penalty=synth.PEN_L1, lam=2.0, tol=1e-9)),
    ("mid_rc_valued_l2", lambda: mid(24, valued=True), [50], [3],
     synth.CoxOptions(penalty=synth.PEN_L2, l2_var=0.5, tol=1e-9)),
    ("mid_cp_l2", lambda: mid(25, counting=True), [20, 60, 120, 180], [1, 7],
     synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9)),
    ("mid_all_tvc", lambda: mid(26, p=6), [10], list(range(6)),
     synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9)),
    ("cuts_outside", lambda: mid(27, p=5), [-5, 500], [2], synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9)),
]
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,make,cuts,tvc,opts", CASES, ids=IDS)
def test_split_fit_matches_oracle(name, make, cuts, tvc, opts):
    d = make()
    with cox.Handle.split(d, cuts, tvc, opts) as h:
        assert h.p == osplit.view_columns(d.p, len(cuts), tvc)[1]
        bg, ig = h.fit()
    sc = osplit.split_counting(d, cuts, tvc)
    bo, io = oracle.fit(sc, opts, max_sweeps=ig["sweeps"])
    assert _rel(bg, bo) <= 1e-9, name
    assert abs(ig["loglik"] - io["loglik"]) <= 1e-11 * abs(io["loglik"])
    if d.start is None and d.n <= 200:
        au = osplit.augment(d, cuts, tvc)
        ba, ia = oracle.fit(au, opts, max_sweeps=ig["sweeps"])
        assert _rel(bg, ba) <= 1e-9


@pytest.mark.parametrize("seed,counting", [(31, False), (32, True)])
def test_split_loglik_matches_definition(seed, counting):
    d = small(seed, counting=counting, valued=True)
    cuts, tvc = [5, 9], [0, 3]
    with cox.Handle.split(d, cuts, tvc) as h:
        rng = np.random.default_rng(seed)
        for _ in range(3):
            b = rng.normal(scale=0.5, size=h.p)
            ref = brute.loglik_step_coef(d, b, cuts, tvc)
            assert h.loglik(b) == pytest.approx(ref, rel=1e-12, abs=1e-12)
            g, hd = h.gradient(b)
            go, ho = oracle.grad_hess(osplit.split_counting(d, cuts, tvc), b)
            assert np.allclose(g, go, rtol=1e-10, atol=1e-10) and np.allclose(hd, ho, rtol=1e-10, atol=1e-10)


def test_split_metadata_is_the_augmented_models():
    """Tie groups (time, stratum id, events, rows at risk) of the view equal those of the
    paper's full augmentation: the rows the view leaves out are never at risk."""
    d = small(33, n=90)
    cuts, tvc = [4, 10], [1]
    au = osplit.augment(d, cuts, tvc)
    with cox.Handle.split(d, cuts, tvc) as h:
        md = h.metadata()
    head, dd, t, k = oracle.tie_groups(au)
    assert md["group_time"].tolist() == t.tolist()
    assert md["group_stratum"].tolist() == k.tolist()
    assert md["group_events"].tolist() == dd.tolist()
    assert md["group_at_risk"].tolist() == oracle.risk_count(au).tolist()


def test_interval_strata_alone_equal_plain_fit():
    """No covariate split: the interval-stratified view gives the unsplit fit (§2.2)."""
    d = mid(34)
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=1.0, tol=1e-10)
    with cox.Handle(d, o) as a, cox.Handle.split(d, [25, 75, 150], [], o) as b:
        ba, ia = a.fit()
        bb, ib = b.fit()
    assert ia["sweeps"] == ib["sweeps"]
    assert _rel(bb, ba) <= 1e-9
    assert abs(ia["loglik"] - ib["loglik"]) <= 1e-11 * abs(ia["loglik"])


def test_treatment_effect_before_and_after_a_cut():
    """The shape of the paper's cough analysis: a treatment whose coefficient steps at day 10,
    L1 on the baseline covariates only (the two treatment copies unpenalized)."""
    rng = np.random.default_rng(35)
    n, p = 6000, 30
    treat = rng.random(n) < 0.5
    x_rows = [np.flatnonzero(treat)] + [np.flatnonzero(rng.random(n) < 0.05) for _ in range(p - 1)]
    early = rng.exponential(40, n)
    late = np.where(treat, rng.exponential(25, n), rng.exponential(45, n))
    t = np.where(early < 10, early, 10 + late)
    stop = np.minimum(np.ceil(t), 120).astype(np.int64)
    event = (t <= 120).astype(np.uint8)
    d = synth.finalize(stop, event, None, None, x_rows, None, p)
    pen = np.ones(p + 1, np.uint8)
    pen[:2] = 0
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=5.0, tol=1e-9, penalize=pen)
    for precision, tb, tl in ((cox.COX_FP64, 1e-9, 1e-11), (cox.COX_FP32C, 1e-5, 1e-7)):
        with cox.Handle.split(d, [10], [0], o, precision=precision) as h:
            bg, ig = h.fit()
        bo, io = oracle.fit(osplit.split_counting(d, [10], [0]), o, max_sweeps=ig["sweeps"])
        assert _rel(bg, bo) <= tb
        assert abs(ig["loglik"] - io["loglik"]) <= tl * abs(io["loglik"])
    assert bo[1] > bo[0] + 0.2     # the treated hazard is higher only after the cut


def test_split_device_inputs():
    import torch
    d = mid(36, counting=True)
    dev = synth.CoxData(**{**d.__dict__})
    for f in ("stop", "start", "event", "stratum", "col_ptr", "row_idx"):
        setattr(dev, f, torch.from_numpy(getattr(d, f)).cuda())
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9)
    with cox.Handle.split(d, [40, 90], [2], o) as a, cox.Handle.split(dev, [40, 90], [2], o) as b:
        ba, ia = a.fit()
        bb, ib = b.fit()
    assert ia["sweeps"] == ib["sweeps"] and _rel(bb, ba) <= 1e-12


@pytest.mark.parametrize("cuts,tvc", [([5, 5], [0]), ([9, 5], [0]), ([5], [4]), ([5], [1, 0]), ([], [0]), ([5], [-1])])
def test_split_rejects_bad_arguments(cuts, tvc):
    d = small(37)
    with pytest.raises(cox.CoxError) as e:
        cox.Handle.split(d, cuts, tvc)
    assert e.value.code == cox.COX_E_INVALID
