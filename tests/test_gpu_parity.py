"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances (FP64 path): integer metadata bit-exact; risk-set sums and log-likelihood 1e-12
relative; gradients 1e-10 (absolute on the 1-scale); fitted beta 1e-9 relative (norm-wise,
max over coordinates / max |beta|) and log-likelihood 1e-11 relative. FP32C path: beta 1e-5,
log-likelihood 1e-7.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import synth
from tests.cases import random_beta, tiny_cases

pytestmark = pytest.mark.gpu

cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def _rel_beta(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if len(b) else 0.0


def _edge_cases():
    out = []
    rng = np.random.default_rng(40)
    # no events at all (G = 0)
    n = 300
    d = synth.finalize(rng.integers(1, 50, n), np.zeros(n, int), None, None,
                       [np.nonzero(rng.random(n) < 0.3)[0] for _ in range(3)], None, 3)
    out.append(("no_events", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0)))
    # every row tied at one time
    n = 5000
    d = synth.finalize(np.full(n, 7), (rng.random(n) < 0.5).astype(int), None, None,
                       [np.nonzero(rng.random(n) < 0.2)[0] for _ in range(4)], None, 4)
    out.append(("all_tied", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=0.5)))
    # size-1 strata (K = n): no risk set has more than one row
    n = 9000
    d = synth.finalize(rng.integers(1, 9, n), (rng.random(n) < 0.5).astype(int), np.arange(n), None,
                       [np.nonzero(rng.random(n) < 0.3)[0] for _ in range(3)], None, 3)
    out.append(("singleton_strata", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0)))
    # a dense all-ones column, an empty column and a one-row column
    n = 12000
    cols = [np.arange(n), np.zeros(0, int), np.array([n // 2]), np.nonzero(rng.random(n) < 0.1)[0]]
    d = synth.finalize(rng.integers(1, 400, n), (rng.random(n) < 0.2).astype(int), rng.integers(0, 5, n), None,
                       cols, None, 4)
    out.append(("odd_columns", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0)))
    # tie heads on tile boundaries: distinct times so that positions 4095/4096/8191/8192 are heads
    n = 8192 * 2 + 77
    stop = np.arange(n) + 1
    ev = np.zeros(n, int)
    ev[[0, 4095, 4096, 8191, 8192, 12287, n - 1]] = 1
    ev[rng.integers(0, n, 200)] = 1
    d = synth.finalize(stop, ev, None, None, [np.nonzero(rng.random(n) < 0.05)[0] for _ in range(3)], None, 3)
    out.append(("tile_boundaries", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0)))
    # more tie groups than a tile can hold (forces head-capped, shortened tiles)
    n = 30000
    d = synth.finalize(np.arange(n) + 1, np.ones(n, int), rng.integers(0, 3, n), None,
                       [np.nonzero(rng.random(n) < 0.05)[0] for _ in range(3)], None, 3)
    out.append(("dense_heads", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0)))
    return out


def _medium_cases():
    out = []
    d, o = synth.stratified_sparse(n=30000, p=24, k=13, n_support=8, event_frac=0.1, dens_lo=0.005, dens_hi=0.2,
                                   admin_days=365, lam_per_n=1e-4, seed=41)
    out.append(("medium_strat_l1", d, o))
    d, o = synth.time_varying(n_subj=8000, p=16, k=4, density=0.05, event_frac=0.3, n_support=6, seed=42)
    out.append(("medium_counting_l2", d, o))
    d, o = synth.plain_dense()
    out.append(("plain_dense_config", d, o))
    return out


CASES = tiny_cases() + _edge_cases() + _medium_cases()
IDS = [c[0] for c in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request):
    name, data, opts = request.param
    h = cox.Handle(data, opts, precision=cox.COX_FP64)
    yield name, data, opts, h
    h.close()


def test_metadata_bit_exact(case):
    name, data, opts, h = case
    md = h.metadata()
    head, dd, t, k = oracle.tie_groups(data)
    assert md["group_time"].tolist() == t.tolist()
    assert md["group_stratum"].tolist() == k.tolist()
    assert md["group_events"].tolist() == dd.tolist()
    assert md["strata_start"].tolist() == oracle.strata(data).tolist()
    s0, _, _ = oracle.risk_sums(data, np.zeros(data.p), -1)
    assert md["group_at_risk"].tolist() == np.rint(s0).astype(np.int64).tolist()
    if data.n <= 2000:
        assert md["group_at_risk"].tolist() == oracle.risk_count(data).tolist()
    dx = h.dx()
    assert np.allclose(dx, oracle.dX(data), rtol=1e-14, atol=0)


def test_risk_sums(case):
    name, data, opts, h = case
    beta = random_beta(data.p, 0.3, seed=3)
    for j in sorted({-1, 0, data.p // 2, data.p - 1}):
        if j >= data.p:
            continue
        S0, S1 = h.risk_sums(beta, j)
        O0, O1, _ = oracle.risk_sums(data, beta, j)
        assert np.allclose(S0, O0, rtol=1e-12, atol=0), (j, np.max(np.abs(S0 - O0) / O0))
        if j >= 0:
            assert np.allclose(S1, O1, rtol=1e-12, atol=1e-300), j


def _ll_scale(data, beta, ll):
    """Magnitude of the terms summed in the log-likelihood: relative error is measured
    against it when the likelihood itself cancels to ~0 (e.g. singleton risk sets)."""
    return max(abs(ll), float(np.abs(beta) @ np.abs(oracle.dX(data))) + float(data.event.sum()))


def test_loglik(case):
    name, data, opts, h = case
    for seed in (0, 5):
        beta = random_beta(data.p, 0.3, seed=seed) if seed else np.zeros(data.p)
        a, b = h.loglik(beta), oracle.loglik(data, beta)
        assert abs(a - b) <= 1e-12 * max(_ll_scale(data, beta, b), 1e-300), (a, b)


def test_gradient_hessian(case):
    name, data, opts, h = case
    beta = random_beta(data.p, 0.3, seed=4)
    g1, g2 = h.gradient(beta)
    o1, o2 = oracle.grad_hess(data, beta)
    assert np.allclose(g1, o1, rtol=1e-10, atol=1e-10 * max(1.0, np.max(np.abs(o1))))
    assert np.allclose(g2, o2, rtol=1e-10, atol=1e-10 * max(1.0, np.max(np.abs(o2))))


def test_fit_fp64(case):
    name, data, opts, h = case
    beta, info = h.fit()
    ob, oinfo = oracle.fit(data, opts, max_sweeps=info["sweeps"])
    assert info["sweeps"] == oinfo["sweeps"] or not oinfo["converged"]
    assert _rel_beta(beta, ob) <= 1e-9, (_rel_beta(beta, ob), info, oinfo)
    assert abs(info["loglik"] - oinfo["loglik"]) <= 1e-11 * max(_ll_scale(data, ob, oinfo["loglik"]), 1e-300)
    if oinfo["converged"]:
        assert info["converged"]


def test_warm_start_and_refit(case):
    """A fit from a warm start follows the oracle from the same start; refits are repeatable."""
    name, data, opts, h = case
    b0 = random_beta(data.p, 0.1, seed=9)
    beta, info = h.fit(b0)
    ob, oinfo = oracle.fit(data, opts, beta0=b0, max_sweeps=info["sweeps"])
    assert _rel_beta(beta, ob) <= 1e-9
    beta2, info2 = h.fit(b0)
    assert _rel_beta(beta2, beta) <= 1e-12 and info2["sweeps"] == info["sweeps"]


@pytest.mark.parametrize("name,data,opts", _medium_cases() + tiny_cases()[:2], ids=lambda x: x if isinstance(x, str) else "")
def test_fit_fp32c(name, data, opts):
    with cox.Handle(data, opts, precision=cox.COX_FP32C) as h:
        beta, info = h.fit()
    ob, oinfo = oracle.fit(data, opts, max_sweeps=info["sweeps"])
    ob2, oinfo2 = oracle.fit(data, opts)
    err = min(_rel_beta(beta, ob), _rel_beta(beta, ob2))
    assert err <= 1e-5, err
    assert abs(info["loglik"] - oinfo2["loglik"]) <= 1e-7 * _ll_scale(data, ob2, oinfo2["loglik"])


def test_batch_matches_single():
    data, o = synth.stratified_sparse(n=20000, p=16, k=9, n_support=6, event_frac=0.1, dens_lo=0.005, dens_hi=0.2,
                                      admin_days=300, seed=50)
    lams = [0.5, 2.0, 8.0, 30.0]
    singles = []
    for lam in lams:
        oo = synth.CoxOptions(penalty=synth.PEN_L1, lam=lam, tol=1e-9)
        with cox.Handle(data, oo) as h:
            singles.append(h.fit())
    base = cox.Handle(data, synth.CoxOptions(penalty=synth.PEN_L1, lam=lams[0], tol=1e-9))
    hs = [base] + [base.clone(synth.CoxOptions(penalty=synth.PEN_L1, lam=lam, tol=1e-9)) for lam in lams[1:]]
    other, oo2 = synth.time_varying(n_subj=3000, p=8, k=2, density=0.1, event_frac=0.3, n_support=3, seed=51)
    hs.append(cox.Handle(other, oo2))
    betas, infos = cox.batch_fit(hs)
    for (b, i), bb, ii in zip(singles, betas, infos):
        assert i["sweeps"] == ii["sweeps"]
        assert _rel_beta(bb, b) <= 1e-12
    ob, oinfo = oracle.fit(other, oo2, max_sweeps=infos[-1]["sweeps"])
    assert _rel_beta(betas[-1], ob) <= 1e-9
    for h in hs:
        h.close()


def test_invalid_inputs_raise():
    d, o = synth.plain_dense(n=50, p=2, seed=1)
    bad = synth.CoxData(**{**d.__dict__})
    bad.stop = d.stop[::-1].copy()
    with pytest.raises(cox.CoxError) as e:
        cox.Handle(bad, o)
    assert e.value.code == cox.COX_E_UNSORTED
    bad = synth.CoxData(**{**d.__dict__})
    bad.event = d.event.copy()
    bad.event[3] = 5
    with pytest.raises(cox.CoxError) as e:
        cox.Handle(bad, o)
    assert e.value.code == cox.COX_E_INVALID
    bad = synth.CoxData(**{**d.__dict__})
    bad.row_idx = d.row_idx.copy()
    bad.row_idx[0] = d.n + 5
    with pytest.raises(cox.CoxError) as e:
        cox.Handle(bad, o)
    assert e.value.code == cox.COX_E_INVALID


def test_device_resident_inputs():
    """Inputs given as torch CUDA tensors (device memory) give the same fit as host arrays."""
    import torch
    d, o = synth.stratified_sparse(n=6000, p=10, k=3, n_support=4, event_frac=0.2, dens_lo=0.01, dens_hi=0.3,
                                   admin_days=100, seed=60)
    dev = synth.CoxData(**{**d.__dict__})
    for f in ("stop", "event", "stratum", "col_ptr", "row_idx"):
        setattr(dev, f, torch.from_numpy(getattr(d, f)).cuda())
    with cox.Handle(d, o) as a, cox.Handle(dev, o) as b:
        ba, ia = a.fit()
        bb, ib = b.fit()
    assert ia["sweeps"] == ib["sweeps"] and _rel_beta(bb, ba) <= 1e-12


@pytest.mark.parametrize("name,data,opts", CASES, ids=IDS)
def test_engines_agree_with_oracle(name, data, opts):
    """The streaming kernel (one launch per coordinate step), the resident kernel (the whole fit
    in one cooperative launch, values held in shared memory) and the incremental kernel (one
    cooperative launch, per-group S0 updated from the changed positions) all follow the oracle's
    CCD path."""
    results = {}
    for eng in (cox.COX_ENGINE_STREAM, cox.COX_ENGINE_RESIDENT, cox.COX_ENGINE_INCR, cox.COX_ENGINE_AUTO):
        with cox.Handle(data, opts, engine=eng) as h:
            try:
                results[eng] = h.fit()
            except cox.CoxError as e:
                assert e.code == cox.COX_E_INVALID and eng in (cox.COX_ENGINE_RESIDENT, cox.COX_ENGINE_INCR), (eng, e)
    for eng, (beta, info) in results.items():
        ob, oinfo = oracle.fit(data, opts, max_sweeps=info["sweeps"])
        assert _rel_beta(beta, ob) <= 1e-9, (eng, _rel_beta(beta, ob))
        assert abs(info["loglik"] - oinfo["loglik"]) <= 1e-11 * _ll_scale(data, ob, oinfo["loglik"]), eng
        assert info["sweeps"] == oinfo["sweeps"] or not oinfo["converged"], eng
    if data.val is None:
        # every binary case here fits the incremental kernel, which AUTO then runs in one launch
        assert cox.COX_ENGINE_INCR in results, name
        assert results[cox.COX_ENGINE_AUTO][1]["step_launches"] == 1
    else:
        assert cox.COX_ENGINE_INCR not in results and cox.COX_ENGINE_RESIDENT not in results


@pytest.mark.parametrize("engine", ["resident", "incr"])
def test_one_launch_engines_reject_valued_x(engine):
    d, o = synth.plain_dense(n=200, p=3, seed=2)
    eng = cox.COX_ENGINE_RESIDENT if engine == "resident" else cox.COX_ENGINE_INCR
    with cox.Handle(d, o, engine=eng) as h:
        with pytest.raises(cox.CoxError) as e:
            h.fit()
    assert e.value.code == cox.COX_E_INVALID


@pytest.mark.parametrize("name,data,opts", _medium_cases()[:2], ids=lambda x: x if isinstance(x, str) else "")
def test_resident_fp32c(name, data, opts):
    with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_RESIDENT) as h:
        beta, info = h.fit()
    assert info["step_launches"] == 1
    ob, oinfo = oracle.fit(data, opts)
    assert _rel_beta(beta, ob) <= 1e-5
    assert abs(info["loglik"] - oinfo["loglik"]) <= 1e-7 * _ll_scale(data, ob, oinfo["loglik"])


def test_resident_then_evaluations_consistent():
    """After a resident fit, the evaluations (which use the streaming kernel on the same state)
    see the written-back values: the gradient at the fitted beta satisfies the KKT conditions."""
    data, o = synth.stratified_sparse(n=40000, p=12, k=7, n_support=5, event_frac=0.1, dens_lo=0.01, dens_hi=0.3,
                                      admin_days=365, seed=77)
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=0.5, tol=1e-14, max_sweeps=500)
    with cox.Handle(data, o) as h:
        beta, info = h.fit()
        assert info["step_launches"] == 1
        g1, _ = h.gradient(beta)
        ll = h.loglik(beta)
    assert np.max(np.abs(g1 + beta / 0.5)) < 1e-6
    assert abs(ll - info["loglik"]) <= 1e-11 * abs(ll)


def test_long_columns_span_segments():
    """Columns longer than one column segment (8192 entries): delta'X of a valued and a binary
    column against the oracle, and an ordering error exactly at a segment boundary rejected."""
    rng = np.random.default_rng(71)
    n = 30000
    stop = np.sort(rng.integers(1, 400, n)).astype(np.int32)
    event = (rng.random(n) < 0.3).astype(np.uint8)
    dense_rows = np.arange(n)
    mid_rows = np.sort(rng.choice(n, 17000, replace=False))
    small_rows = np.sort(rng.choice(n, 40, replace=False))
    rows = [dense_rows, mid_rows, small_rows, np.zeros(0, np.int64)]
    vals = [rng.normal(size=len(r)) for r in rows]
    d = synth.finalize(stop, event, None, None, rows, vals, 4)
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-10)
    with cox.Handle(d, o) as h:
        assert np.allclose(h.dx(), oracle.dX(d), rtol=1e-12, atol=1e-12)
        bh, ih = h.fit()
    bo, io = oracle.fit(d, o, max_sweeps=ih["sweeps"])
    assert _rel_beta(bh, bo) <= 1e-9
    db = synth.finalize(stop, event, None, None, rows, None, 4)
    with cox.Handle(db, o) as h:
        assert h.dx().tolist() == oracle.dX(db).tolist()
    bad = synth.CoxData(**{**db.__dict__})
    bad.row_idx = db.row_idx.copy()
    a = int(db.col_ptr[1])
    bad.row_idx[a + 8192] = bad.row_idx[a + 8191]   # first entry of the column's second segment
    with pytest.raises(cox.CoxError) as e:
        cox.Handle(bad, o)
    assert e.value.code == cox.COX_E_INVALID


@pytest.mark.parametrize("k", [1, 40, 1500])
def test_paper_synthetic_shape(k):
    """The shape of the paper's synthetic experiment (5 % binary X, 20 % of beta nonzero,
    L1 gamma = sqrt 2) from one stratum to strata of two rows: the GPU fit follows the oracle."""
    d, o = synth.synthetic_e1(n=3000, p=40, k=k, seed=81)
    with cox.Handle(d, o) as h:
        b, info = h.fit()
    ob, oi = oracle.fit(d, o, max_sweeps=info["sweeps"])
    assert _rel_beta(b, ob) <= 1e-9
    assert abs(info["loglik"] - oi["loglik"]) <= 1e-11 * max(abs(oi["loglik"]), 1.0)
