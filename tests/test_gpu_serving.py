"""The continuous-batching server (cox_server_*): results in the mix equal standalone fits on
the engine the server gives each request (the incremental kernel when its data qualify, else the
streaming work list), admission by memory footprint, cancellation."""
from __future__ import annotations

import threading

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import synth

pytestmark = pytest.mark.gpu
cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def _requests():
    out = []
    for i in range(6):
        d, o = synth.stratified_sparse(n=3000 + 4000 * i, p=6 + 3 * i, k=1 + 5 * i, n_support=3, event_frac=0.2,
                                       dens_lo=0.01, dens_hi=0.3, admin_days=200, lam_per_n=3e-4, seed=100 + i)
        out.append((d, o))
    for i in range(4):
        d, o = synth.time_varying(n_subj=1500 + 1000 * i, p=5 + 2 * i, k=1 + i, density=0.05, event_frac=0.3,
                                  n_support=3, seed=200 + i)
        out.append((d, o))
    d, o = synth.plain_dense(n=500, p=5, seed=300)
    out.append((d, o))
    return out


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _alone(d, o, precision=cox.COX_FP64):
    """The request fitted on its own by the engine the server gives it: the incremental kernel
    when the data qualify for it, else the streaming kernel."""
    with cox.Handle(d, o, precision=precision) as h:
        r = h.fit()
    if r[1]["engine"] == cox.COX_ENGINE_INCR:
        return r
    with cox.Handle(d, o, precision=precision, engine=cox.COX_ENGINE_STREAM) as h:
        return h.fit()


def test_results_in_the_mix_equal_standalone_fits():
    reqs = _requests()
    alone = [_alone(d, o) for d, o in reqs]
    # a budget that holds only a few requests at once, so that the queue, admission and
    # retirement all take part while the other fits are in flight
    budget = 6 * max(cox.cox_footprint(d, o) for d, o in reqs)
    with cox.Server(memory_budget=budget, max_active=5) as srv:
        ids = [srv.submit(d, o) for d, o in reqs]
        got = [srv.wait(i, 120.0) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["running"] == 0
    for (b, info), (bb, ii), (d, o) in zip(alone, got, reqs):
        assert ii["sweeps"] == info["sweeps"] and ii["converged"] == info["converged"]
        assert _rel(bb, b) <= 1e-12, (d.recipe, _rel(bb, b))
        assert abs(ii["loglik"] - info["loglik"]) <= 1e-12 * abs(info["loglik"])
        assert ii["total_ms"] >= ii["wait_ms"] >= 0.0


def test_concurrent_submitters_and_polling():
    reqs = _requests()[:6]
    results = {}
    with cox.Server(max_active=3) as srv:
        def worker(k):
            d, o = reqs[k]
            rid = srv.submit(d, o)
            while True:
                r = srv.poll(rid)
                if r is not None:
                    results[k] = r
                    return
        th = [threading.Thread(target=worker, args=(k,)) for k in range(len(reqs))]
        for t in th:
            t.start()
        for t in th:
            t.join(120)
    assert len(results) == len(reqs)
    for k, (d, o) in enumerate(reqs):
        b, info = _alone(d, o)
        assert _rel(results[k][0], b) <= 1e-12


def test_admission_rejects_requests_above_the_budget_and_cancel_frees():
    d, o = synth.stratified_sparse(n=20000, p=8, k=3, n_support=3, event_frac=0.2, dens_lo=0.01, dens_hi=0.3,
                                   admin_days=200, seed=5)
    fp = cox.cox_footprint(d, o)
    with cox.Server(memory_budget=fp // 2) as srv:
        with pytest.raises(cox.CoxError) as e:
            srv.submit(d, o)
        assert e.value.code == cox.COX_E_ADMISSION
    with cox.Server(memory_budget=4 * fp, max_active=1) as srv:
        a = srv.submit(d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=0.0, max_sweeps=1_000_000))
        b = srv.submit(d, o)
        srv.cancel(a)
        with pytest.raises(cox.CoxError):
            srv.wait(a, 60.0)
        rb = srv.wait(b, 60.0)
        assert rb is not None and rb[1]["converged"]
        st = srv.stats()
        assert st["bytes_in_use"] == 0 and st["running"] == 0


def _ll_scale(data, beta, ll):
    """Magnitude of the terms summed in the log-likelihood (the relative error's denominator)."""
    return max(abs(ll), float(np.abs(beta) @ np.abs(oracle.dX(data))) + float(data.event.sum()))


@pytest.mark.parametrize("precision,btol,ltol", [(cox.COX_FP64, 1e-9, 1e-11), (cox.COX_FP32C, 1e-5, 1e-7)],
                         ids=["fp64", "fp32c"])
def test_served_results_match_the_oracle(precision, btol, ltol):
    """Every result the server returns, with the other requests in flight beside it, is the
    oracle's fit of that request after the same number of sweeps, within the path's tolerance
    (FP64: 1e-9 in beta, 1e-11 in the log-likelihood; compensated FP32: 1e-5 and 1e-7)."""
    reqs = _requests()
    budget = 6 * max(cox.cox_footprint(d, o, precision) for d, o in reqs)
    with cox.Server(memory_budget=budget, max_active=5, precision=precision) as srv:
        ids = [srv.submit(d, o) for d, o in reqs]
        got = [srv.wait(i, 120.0) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    for (bb, ii), (d, o) in zip(got, reqs):
        if precision == cox.COX_FP64:
            ob, oi = oracle.fit(d, o, max_sweeps=ii["sweeps"])
            assert ii["sweeps"] == oi["sweeps"] or not oi["converged"], (d.recipe, ii, oi)
        else:
            # the convergence test of a compensated-FP32 fit may fall one sweep apart from the
            # FP64 oracle's; the iterates are compared after the same number of sweeps
            o_same = synth.CoxOptions(penalty=o.penalty, lam=o.lam, l2_var=o.l2_var, penalize=o.penalize, tol=0.0)
            ob, oi = oracle.fit(d, o_same, max_sweeps=ii["sweeps"])
        assert _rel(bb, ob) <= btol, (d.recipe, _rel(bb, ob))
        assert abs(ii["loglik"] - oi["loglik"]) <= ltol * _ll_scale(d, ob, oi["loglik"]), (d.recipe, ii, oi)


def test_fp32c_results_in_the_mix_equal_standalone_fits():
    """The compensated-FP32 server: each result in the mix equals the same request fitted alone
    with the same precision, within the stated FP32C tolerance (1e-5 in beta, 1e-7 in the
    log-likelihood)."""
    reqs = _requests()
    alone = [_alone(d, o, cox.COX_FP32C) for d, o in reqs]
    budget = 6 * max(cox.cox_footprint(d, o, cox.COX_FP32C) for d, o in reqs)
    with cox.Server(memory_budget=budget, max_active=5, precision=cox.COX_FP32C) as srv:
        ids = [srv.submit(d, o) for d, o in reqs]
        got = [srv.wait(i, 120.0) for i in ids]
    for (b, info), (bb, ii), (d, o) in zip(alone, got, reqs):
        assert abs(ii["sweeps"] - info["sweeps"]) <= 1, (d.recipe, ii, info)
        assert _rel(bb, b) <= 1e-5, (d.recipe, _rel(bb, b))
        assert abs(ii["loglik"] - info["loglik"]) <= 1e-7 * _ll_scale(d, b, info["loglik"])


def _mixed_size_requests():
    """Requests of several sizes with binary X: the server runs each whole on the incremental
    kernel (between replays of its work list) when its data qualify, else in the work list."""
    out = _requests()[:4]
    d, o = synth.stratified_sparse(n=300_000, p=8, k=20, n_support=4, event_frac=0.1, dens_lo=0.005, dens_hi=0.2,
                                   admin_days=400, lam_per_n=1e-4, seed=400)
    out.append((d, o))
    d, o = synth.time_varying(n_subj=60_000, p=6, k=4, density=0.05, event_frac=0.3, n_support=3, seed=401)
    out.append((d, o))
    return out


@pytest.mark.parametrize("precision,btol,ltol", [(cox.COX_FP64, 1e-9, 1e-11), (cox.COX_FP32C, 1e-5, 1e-7)],
                         ids=["fp64", "fp32c"])
def test_large_requests_run_on_the_incremental_kernel_and_match_the_oracle(precision, btol, ltol):
    reqs = _mixed_size_requests()
    with cox.Server(max_active=4, precision=precision) as srv:
        ids = [srv.submit(d, o) for d, o in reqs]
        got = [srv.wait(i, 300.0) for i in ids]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["running"] == 0 and st["bytes_in_use"] == 0
    for (bb, ii), (d, o) in zip(got, reqs):
        with cox.Handle(d, o, precision=precision) as h:   # AUTO: the engine the data qualify for
            _, alone = h.fit()
        want = cox.COX_ENGINE_INCR if alone["engine"] == cox.COX_ENGINE_INCR else cox.COX_ENGINE_STREAM
        assert ii["engine"] == want, (d.recipe, ii["engine"], alone["engine"])
        o_same = synth.CoxOptions(penalty=o.penalty, lam=o.lam, l2_var=o.l2_var, penalize=o.penalize, tol=0.0)
        ob, oi = oracle.fit(d, o_same, max_sweeps=ii["sweeps"])
        assert _rel(bb, ob) <= btol, (d.recipe, _rel(bb, ob))
        assert abs(ii["loglik"] - oi["loglik"]) <= ltol * _ll_scale(d, ob, oi["loglik"]), (d.recipe, ii, oi)
