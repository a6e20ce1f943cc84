"""Parity at the full benchmark sizes, in the engine the benchmark uses, on sampled outputs the
oracle can compute one by one: risk-set sums, log-likelihood and derivatives at a random beta for
a few sampled coordinates, and the optimality conditions of the GPU fit checked by the oracle.
Tolerances as in the small-size parity tests: FP64 sums and log-likelihood 1e-12, derivatives
1e-10 on their own scale; FP32C sums 1e-6, log-likelihood 1e-7, derivatives 1e-5."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import synth

pytestmark = pytest.mark.gpu
cox = pytest.importorskip("paper_2310_16238_gb300.cox")


@pytest.fixture(scope="module")
def stratified_full():
    return synth.stratified_sparse()          # N = 2e6, p = 2000, K = 100 (the bench workload)


@pytest.fixture(scope="module")
def counting_full():
    return synth.time_varying()               # 1e6 subjects, ~2.9e6 rows, p = 5000, K = 20


def _magnitudes(data, beta, j):
    """Sum over all rows of exp(eta) and of |x_j| exp(eta): the scale that bounds the rounding
    error of a risk-set sum whose entries and exits cancel (counting-process rows)."""
    D = np.exp(oracle.eta(data, beta))
    a, b = data.col_ptr[j], data.col_ptr[j + 1]
    x = np.ones(b - a) if data.val is None else np.abs(data.val[a:b])
    return float(D.sum()), float(np.sum(x * D[data.row_idx[a:b]]))


def _sampled_parity(data, opts, precision, rtol_sum, rtol_ll, rtol_g):
    rng = np.random.default_rng(1)
    beta = np.zeros(data.p)
    sup = rng.choice(data.p, 40, replace=False)
    beta[sup] = rng.normal(0, 0.2, 40)
    cols = [int(c) for c in rng.choice(data.p, 3, replace=False)] + [int(sup[0])]
    dX = oracle.dX(data)
    with cox.Handle(data, opts, precision=precision) as h:
        ll, oll = h.loglik(beta), oracle.loglik(data, beta)
        assert abs(ll - oll) <= rtol_ll * _ll_scale(data, beta, oll), (ll, oll)
        g1, g2 = h.gradient(beta)
        o1, o2 = oracle.grad_hess(data, beta, cols)
        for k, j in enumerate(cols):
            scale = max(1.0, abs(o1[k]), abs(dX[j]), abs(o2[k]))
            assert abs(g1[j] - o1[k]) <= rtol_g * scale, (j, g1[j], o1[k])
            assert abs(g2[j] - o2[k]) <= rtol_g * scale, (j, g2[j], o2[k])
        j = cols[0]
        S0, S1 = h.risk_sums(beta, j)
        O0, O1, _ = oracle.risk_sums(data, beta, j)
        t0, t1 = _magnitudes(data, beta, j) if data.start is not None else (0.0, 0.0)
        assert np.all(np.abs(S0 - O0) <= rtol_sum * (np.abs(O0) + t0))
        assert np.all(np.abs(S1 - O1) <= rtol_sum * (np.abs(O1) + t1))
        bfit, info = h.fit()   # the engine the benchmark runs (AUTO: incremental for binary X)
        assert info["converged"] and info["step_launches"] == 1
    return bfit, info


def _other_engine_agrees(data, opts, beta, info, engine, tol):
    """The same fit through another engine (independent kernels) lands on the same path."""
    with cox.Handle(data, opts, engine=engine) as h:
        b2, i2 = h.fit()
    assert i2["sweeps"] == info["sweeps"]
    assert np.max(np.abs(b2 - beta)) <= tol * max(np.max(np.abs(b2)), 1e-300)


def _ll_scale(data, beta, ll):
    """Magnitude of the terms the log-likelihood sums: |loglik|, sum |beta_j dX_j| and the events."""
    dX = oracle.dX(data)
    return max(abs(ll), float(np.sum(np.abs(beta * dX))) + float(np.sum(data.event)))


def _kkt(data, opts, beta, objective, cols):
    """KKT conditions of the penalized objective at the GPU fit, with the oracle's derivatives.

    The fit stopped when a whole sweep lowered the objective by at most tol*|objective|; a
    coordinate whose optimality residual is r would lower it by about r^2 / (2 g'') in one
    Newton step, so r is bounded by sqrt(2 g'' tol |objective|) (times a safety factor 10)."""
    g1, g2 = oracle.grad_hess(data, beta, cols)
    for k, j in enumerate(cols):
        bound = 10.0 * np.sqrt(2.0 * g2[k] * opts.tol * abs(objective)) + 1e-9 * max(1.0, abs(g1[k]))
        if opts.penalty == synth.PEN_L2:
            assert abs(g1[k] + beta[j] / opts.l2_var) <= bound, (j, g1[k], beta[j], bound)
        elif beta[j] != 0.0:
            assert abs(g1[k] + np.sign(beta[j]) * opts.lam) <= bound, (j, g1[k], beta[j], bound)
        else:
            assert abs(g1[k]) <= opts.lam + bound, (j, g1[k], bound)


def test_stratified_full_size_fp64(stratified_full):
    data, opts = stratified_full
    beta, info = _sampled_parity(data, opts, cox.COX_FP64, 1e-12, 1e-12, 1e-10)
    _other_engine_agrees(data, opts, beta, info, cox.COX_ENGINE_RESIDENT, 1e-9)
    # the bench's L1 weight keeps every coefficient at 0: check that the oracle agrees
    cols = list(range(0, data.p, 97))
    _kkt(data, opts, beta, info["objective"], cols)
    # a weaker penalty moves coefficients: KKT of the GPU fit checked by the oracle
    o2 = synth.CoxOptions(penalty=synth.PEN_L1, lam=1e-5 * data.n, tol=1e-12)
    with cox.Handle(data, o2) as h:
        b2, i2 = h.fit()
        assert i2["step_launches"] == 1
        assert abs(h.loglik(b2) - oracle.loglik(data, b2)) <= 1e-11 * _ll_scale(data, b2, i2["loglik"])
    assert i2["converged"] and np.count_nonzero(b2) > 0
    moved = [int(j) for j in np.nonzero(b2)[0][:4]] + cols[:3]
    _kkt(data, o2, b2, i2["objective"], moved)


def test_stratified_full_size_fp32c(stratified_full):
    data, opts = stratified_full
    _sampled_parity(data, opts, cox.COX_FP32C, 1e-6, 1e-7, 1e-5)


def test_counting_full_size_fp64(counting_full):
    data, opts = counting_full
    beta, info = _sampled_parity(data, opts, cox.COX_FP64, 1e-12, 1e-12, 1e-10)
    _other_engine_agrees(data, opts, beta, info, cox.COX_ENGINE_STREAM, 1e-9)
    _kkt(data, opts, beta, info["objective"], [0, 1, 2, int(np.argmax(np.abs(beta)))])


def _first_columns(data, p):
    """The same rows with only the first p columns of X."""
    end = int(data.col_ptr[p])
    return synth.CoxData(**{**data.__dict__, "p": p, "col_ptr": data.col_ptr[:p + 1].copy(),
                            "row_idx": data.row_idx[:end], "val": None if data.val is None else data.val[:end]})


def _iterate_parity(data, opts, sweeps, precision, engine, btol, ltol, oracle_fit=None):
    """The GPU fit after `sweeps` sweeps against the oracle's after the same sweeps, element by
    element: beta (relative, norm-wise) and the fit's own reported log-likelihood."""
    o = synth.CoxOptions(penalty=opts.penalty, lam=opts.lam, l2_var=opts.l2_var, penalize=opts.penalize, tol=0.0,
                         max_sweeps=sweeps)
    with cox.Handle(data, o, precision=precision, engine=engine) as h:
        b, info = h.fit()
    ob, oi = oracle_fit if oracle_fit is not None else oracle.fit(data, o, max_sweeps=sweeps)
    assert info["sweeps"] == oi["sweeps"] == sweeps, (info, oi)
    err_b = float(np.max(np.abs(b - ob)) / max(np.max(np.abs(ob)), 1e-300))
    err_l = abs(info["loglik"] - oi["loglik"]) / _ll_scale(data, ob, oi["loglik"])
    assert err_b <= btol and err_l <= ltol, (err_b, err_l, info, oi)
    return (ob, oi), info


def test_stratified_moving_fit_matches_the_oracle(stratified_full):
    """The benchmark's workload (N = 2e6, p = 2000, K = 100) at the weaker L1 weight 1e-5 N, where
    hundreds of coefficients move and every step's eta / exp(eta) update runs: after two sweeps
    the AUTO engine (the incremental kernel, double-word sums) equals the oracle to 1e-9 in beta
    and 1e-11 in its own reported log-likelihood, element by element."""
    data, opts = stratified_full
    o = synth.CoxOptions(penalty=synth.PEN_L1, lam=1e-5 * data.n)
    (ob, oi), info = _iterate_parity(data, o, 2, cox.COX_FP64, cox.COX_ENGINE_AUTO, 1e-9, 1e-11)
    assert info["engine"] == cox.COX_ENGINE_INCR and np.count_nonzero(ob) > 100
    # the dense streaming kernel on the same iterates, in FP64 and in compensated FP32
    _iterate_parity(data, o, 2, cox.COX_FP64, cox.COX_ENGINE_STREAM, 1e-9, 1e-11, (ob, oi))
    _iterate_parity(data, o, 2, cox.COX_FP32C, cox.COX_ENGINE_STREAM, 1e-5, 1e-7, (ob, oi))


def test_counting_full_rows_first_columns_match_the_oracle(counting_full):
    """The counting-process workload at its full size in rows (1e6 subjects, ~2.9e6 (start, stop]
    rows, 5.8e6 risk positions, K = 20) with its first 200 columns: after two sweeps the AUTO
    engine equals the oracle to 1e-9 / 1e-11, the streaming kernel in compensated FP32 to 1e-5 /
    1e-7."""
    data, opts = counting_full
    sub = _first_columns(data, 200)
    (ob, oi), info = _iterate_parity(sub, opts, 2, cox.COX_FP64, cox.COX_ENGINE_AUTO, 1e-9, 1e-11)
    assert np.count_nonzero(ob) > 0.9 * sub.p
    _iterate_parity(sub, opts, 2, cox.COX_FP32C, cox.COX_ENGINE_STREAM, 1e-5, 1e-7, (ob, oi))
