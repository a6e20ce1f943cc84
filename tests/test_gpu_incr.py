"""The incremental kernel (per-group S0 kept resident, updated from the changed positions, one
cooperative launch per fit) against the oracle on cases aimed at its own logic: strata that span
many CTAs, CTAs holding many stratum ends, counting-process rows whose entry and exit fall in
different CTAs, one and two columns, the sweep limit, warm starts and the state left for the
evaluations. Tolerances as in the other parity tests (FP64: beta 1e-9, log-likelihood 1e-11;
FP32C: beta 1e-5, log-likelihood 1e-7)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import synth
from tests.cases import random_beta

pytestmark = pytest.mark.gpu
cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if len(b) else 0.0


def _ll_scale(data, beta, ll):
    dX = oracle.dX(data)
    return max(abs(ll), float(np.sum(np.abs(beta * dX))) + float(np.sum(data.event)))


def _cases():
    out = []
    # one big stratum spread over every CTA, plus small ones
    d, o = synth.stratified_sparse(n=150000, p=12, k=6, n_support=6, event_frac=0.1, dens_lo=0.002, dens_hi=0.2,
                                   admin_days=2000, lam_per_n=1e-4, seed=61)
    out.append(("wide_strata_l1", d, o))
    # many small strata: most CTAs hold several stratum ends
    d, o = synth.stratified_sparse(n=60000, p=8, k=3000, n_support=4, event_frac=0.3, dens_lo=0.02, dens_hi=0.3,
                                   admin_days=100, lam_per_n=1e-4, seed=62)
    out.append(("many_strata_l1", d, o))
    # counting-process rows, L2
    d, o = synth.time_varying(n_subj=30000, p=10, k=3, density=0.02, event_frac=0.3, n_support=5, seed=63)
    out.append(("counting_l2", d, o))
    # one column and two columns
    d, o = synth.stratified_sparse(n=20000, p=1, k=4, n_support=1, event_frac=0.2, dens_lo=0.2, dens_hi=0.3,
                                   admin_days=300, lam_per_n=0.0, seed=64)
    out.append(("one_column", d, synth.CoxOptions(penalty=synth.PEN_NONE, tol=1e-12)))
    d, o = synth.time_varying(n_subj=5000, p=2, k=2, density=0.3, event_frac=0.4, n_support=2, seed=65)
    out.append(("two_columns_counting", d, o))
    return out


CASES = _cases()
IDS = [c[0] for c in CASES]


@pytest.mark.parametrize("name,data,opts", CASES, ids=IDS)
def test_incr_fit_matches_oracle(name, data, opts):
    with cox.Handle(data, opts, engine=cox.COX_ENGINE_INCR) as h:
        beta, info = h.fit()
        assert info["step_launches"] == 1
        # the state the kernel leaves behind is what the evaluations see
        ll = h.loglik(beta)
    ob, oinfo = oracle.fit(data, opts, max_sweeps=info["sweeps"])
    assert info["sweeps"] == oinfo["sweeps"] or not oinfo["converged"]
    assert _rel(beta, ob) <= 1e-9, _rel(beta, ob)
    scale = _ll_scale(data, ob, oinfo["loglik"])
    assert abs(info["loglik"] - oinfo["loglik"]) <= 1e-11 * scale
    assert abs(ll - info["loglik"]) <= 1e-11 * scale


@pytest.mark.parametrize("name,data,opts", CASES[:3], ids=IDS[:3])
def test_incr_sweep_limit_and_warm_start(name, data, opts):
    o = synth.CoxOptions(penalty=opts.penalty, lam=opts.lam, l2_var=opts.l2_var, tol=1e-14, max_sweeps=2)
    b0 = random_beta(data.p, 0.05, seed=3)
    with cox.Handle(data, o, engine=cox.COX_ENGINE_INCR) as h:
        beta, info = h.fit(b0)
    assert info["sweeps"] == 2 and not info["converged"] and info["rc"] == cox.COX_W_NOT_CONVERGED
    ob, oinfo = oracle.fit(data, o, beta0=b0, max_sweeps=2)
    assert _rel(beta, ob) <= 1e-9
    assert abs(info["loglik"] - oinfo["loglik"]) <= 1e-11 * _ll_scale(data, ob, oinfo["loglik"])


@pytest.mark.parametrize("name,data,opts", CASES[:3], ids=IDS[:3])
def test_incr_fp32c(name, data, opts):
    with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_INCR) as h:
        beta, info = h.fit()
    ob, oinfo = oracle.fit(data, opts)
    assert _rel(beta, ob) <= 1e-5
    assert abs(info["loglik"] - oinfo["loglik"]) <= 1e-7 * _ll_scale(data, ob, oinfo["loglik"])


def test_incr_is_deterministic_and_matches_streaming():
    name, data, opts = CASES[0]
    with cox.Handle(data, opts, engine=cox.COX_ENGINE_INCR) as h:
        b1, i1 = h.fit()
        b2, i2 = h.fit()
    assert np.array_equal(b1, b2) and i1["loglik"] == i2["loglik"]
    with cox.Handle(data, opts, engine=cox.COX_ENGINE_STREAM) as h:
        b3, i3 = h.fit()
    assert i3["sweeps"] == i1["sweeps"] and _rel(b1, b3) <= 1e-10


def test_incr_batch_waves_match_oracle():
    """A batch on the incremental kernel: each fit on its own compact plan, fits packed into
    waves of at most one CTA per SM (this batch needs more than one wave), warm starts included."""
    sets = []
    d1, _ = synth.stratified_sparse(n=150000, p=10, k=6, n_support=5, event_frac=0.1, dens_lo=0.005, dens_hi=0.2,
                                    admin_days=2000, seed=71)
    sets += [(d1, synth.CoxOptions(penalty=synth.PEN_L1, lam=lam, tol=1e-10)) for lam in np.geomspace(5.0, 500.0, 24)]
    d2, o2 = synth.time_varying(n_subj=8000, p=8, k=3, density=0.05, event_frac=0.3, n_support=4, seed=72)
    sets += [(d2, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=v, tol=1e-10)) for v in (0.1, 1.0, 10.0)]
    d3, _ = synth.stratified_sparse(n=3000, p=5, k=40, n_support=3, event_frac=0.4, dens_lo=0.05, dens_hi=0.5,
                                    admin_days=50, seed=73)
    sets += [(d3, synth.CoxOptions(penalty=synth.PEN_L1, lam=1.0, tol=1e-10))]
    handles, by_data = [], {}
    for d, o in sets:
        if id(d) in by_data:
            handles.append(by_data[id(d)].clone(o))
        else:
            h = cox.Handle(d, o)
            by_data[id(d)] = h
            handles.append(h)
    b0 = [None] * len(sets)
    b0[-1] = random_beta(sets[-1][0].p, 0.05, seed=2)
    betas, infos = cox.batch_fit(handles, [np.zeros(d.p) if b is None else b for (d, _), b in zip(sets, b0)])
    try:
        for (d, o), b, beta, info in zip(sets, b0, betas, infos):
            assert info["engine"] == cox.COX_ENGINE_INCR and info["step_launches"] == 1
            ob, oinfo = oracle.fit(d, o, beta0=b, max_sweeps=info["sweeps"])
            assert info["sweeps"] == oinfo["sweeps"] or not oinfo["converged"]
            assert _rel(beta, ob) <= 1e-9, _rel(beta, ob)
            assert abs(info["loglik"] - oinfo["loglik"]) <= 1e-11 * _ll_scale(d, ob, oinfo["loglik"])
    finally:
        for h in handles:
            h.close()


def _dense_column_data(n, dense_cols, p=10, seed=70, n_strata=3, counting=False):
    """Sparse binary columns plus the listed columns held by about half the rows (a treatment
    indicator): too dense for the incremental lists of any plan on one CTA per SM."""
    rng = np.random.default_rng(seed)
    stop = rng.integers(1, 400, n)
    event = (rng.random(n) < 0.2).astype(np.uint8)
    stratum = rng.integers(0, n_strata, n)
    start = (stop - rng.integers(1, 80, n)) if counting else None
    rows = []
    for j in range(p):
        dens = 0.5 if j in dense_cols else float(np.exp(rng.uniform(np.log(0.002), np.log(0.05))))
        rows.append(np.flatnonzero(rng.random(n) < dens))
    return synth.finalize(stop, event, stratum, start, rows, None, p)


@pytest.mark.parametrize("dense_cols,counting,pen", [
    ([3], False, "l1"), ([0, 1], False, "l2"), ([9], True, "l2"), ([0, 4, 47], False, "l1"),
], ids=["one_mid_l1", "two_first_l2", "last_counting_l2", "three_l1"])
def test_incr_hands_dense_columns_to_the_resident_kernel(dense_cols, counting, pen):
    # at most max(2, p / 16) columns are handed over; more than that and the fit stays resident
    d = _dense_column_data(420000 if not counting else 220000, dense_cols, p=10 if len(dense_cols) < 3 else 48,
                           counting=counting)
    o = (synth.CoxOptions(penalty=synth.PEN_L1, lam=20.0, tol=1e-9) if pen == "l1"
         else synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9))
    with cox.Handle(d, o) as h:
        beta, info = h.fit()
        ll_eval = h.loglik(beta)
    assert info["engine"] == cox.COX_ENGINE_INCR
    assert info["step_launches"] > 2            # launches alternate at the dense columns
    ob, oi = oracle.fit(d, o, max_sweeps=info["sweeps"])
    assert _rel(beta, ob) <= 1e-9
    scale = _ll_scale(d, ob, oi["loglik"])
    assert abs(info["loglik"] - oi["loglik"]) <= 1e-11 * scale
    assert abs(ll_eval - oracle.loglik(d, beta)) <= 1e-11 * scale
    with cox.Handle(d, o, engine=cox.COX_ENGINE_RESIDENT) as h:
        br, ir = h.fit()
    assert ir["sweeps"] == info["sweeps"] and _rel(beta, br) <= 1e-9


def test_too_many_dense_columns_stay_resident():
    d = _dense_column_data(420000, [0, 4, 9], p=10)
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9)
    with cox.Handle(d, o) as h:
        beta, info = h.fit()
    assert info["engine"] == cox.COX_ENGINE_RESIDENT
    ob, oi = oracle.fit(d, o, max_sweeps=info["sweeps"])
    assert _rel(beta, ob) <= 1e-9


def test_dense_column_hand_over_fp32c():
    d = _dense_column_data(420000, [2], p=10, seed=71)
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-9)
    with cox.Handle(d, o, precision=cox.COX_FP32C) as h:
        beta, info = h.fit()
    assert info["engine"] == cox.COX_ENGINE_INCR and info["step_launches"] > 2
    ob, oi = oracle.fit(d, o, max_sweeps=info["sweeps"])
    assert _rel(beta, ob) <= 1e-5
    assert abs(info["loglik"] - oi["loglik"]) <= 1e-7 * _ll_scale(d, ob, oi["loglik"])


@pytest.mark.parametrize("precision,tb,tl", [(cox.COX_FP64, 1e-9, 1e-11), (cox.COX_FP32C, 1e-5, 1e-7)],
                         ids=["fp64", "fp32c"])
def test_group_dense_configuration(precision, tb, tl):
    """More tie groups than one per thread of every CTA (the shape of the paper's synthetic
    experiment with many strata): the configuration with up to four groups per thread."""
    d, o = synth.synthetic_e1(n=300000, p=24, k=30000, seed=90)
    G = len(oracle.tie_groups(d)[0])
    assert G > 1024 * 152            # beyond one group per thread on every SM
    with cox.Handle(d, o, precision=precision) as h:
        beta, info = h.fit()
    assert info["engine"] == cox.COX_ENGINE_INCR and info["step_launches"] == 1
    ob, oi = oracle.fit(d, o, max_sweeps=info["sweeps"])
    assert _rel(beta, ob) <= tb
    assert abs(info["loglik"] - oi["loglik"]) <= tl * _ll_scale(d, ob, oi["loglik"])
