"""Pins for the CPU oracle (no GPU): worked example, brute force, closed forms, finite
differences, textbook special cases and the paper's model-equivalence invariants."""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import synth
from tests import brute
from tests.cases import random_beta, tiny_cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        out[k] = [float(x) for x in v]
    return out


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))) if a.size else 0.0


# ------------------------------------------------------------------ §2.6 worked example
def test_segscan_paper_example():
    g = _golden_kv("segscan_p704.txt")
    b = oracle.segscan(g["a"], np.array(g["f"], dtype=np.uint8))
    assert b.tolist() == g["b"]


def test_segscan_matches_sequential_definition():
    rng = np.random.default_rng(5)
    for n in (1, 2, 17, 300):
        a = rng.integers(-5, 9, n).astype(float)
        f = (rng.random(n) < 0.2).astype(np.uint8)
        f[0] = 1
        b = oracle.segscan(a, f)
        ref, acc = [], 0.0
        for i in range(n):
            acc = a[i] if f[i] else acc + a[i]
            ref.append(acc)
        assert b.tolist() == ref


# ------------------------------------------------------------------ integer metadata
@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_tie_groups_and_risk_counts(name, data, opts):
    head, d, t, k = oracle.tie_groups(data)
    bg = brute.groups(data)
    assert [(int(a), int(b), int(c)) for a, b, c in zip(k, t, d)] == bg
    for g in range(len(head)):
        r = head[g]
        kk = 0 if data.stratum is None else data.stratum[r]
        assert data.stop[r] == t[g] and kk == k[g]
        assert r == 0 or data.stop[r - 1] != t[g] or (data.stratum is not None and data.stratum[r - 1] != kk)
    assert oracle.risk_count(data).tolist() == brute.risk_count(data).tolist()


@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_strata_offsets(name, data, opts):
    off = oracle.strata(data)
    s = np.zeros(data.n, np.int64) if data.stratum is None else data.stratum
    starts = [0] + [r for r in range(1, data.n) if s[r] != s[r - 1]]
    assert off.tolist() == starts + [data.n]


def test_validate_rejects_bad_input():
    d, _ = synth.plain_dense(n=30, p=2, seed=3)
    assert oracle.validate(d) == 0
    bad = synth.CoxData(**{**d.__dict__})
    bad.stop = d.stop[::-1].copy()
    assert oracle.validate(bad) == -2
    bad = synth.CoxData(**{**d.__dict__})
    bad.event = d.event.copy(); bad.event[0] = 2
    assert oracle.validate(bad) == -1


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_risk_sums_vs_brute(name, data, opts):
    beta = random_beta(data.p, 0.4, seed=1)
    for j in [-1] + list(range(data.p)):
        S = oracle.risk_sums(data, beta, j)
        B = brute.risk_sums(data, beta, j)
        for s, b in zip(S, B):
            assert np.allclose(s, b, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_loglik_grad_hess_vs_brute(name, data, opts):
    beta = random_beta(data.p, 0.4, seed=2)
    assert abs(oracle.loglik(data, beta) - brute.loglik(data, beta)) <= 1e-12 * abs(brute.loglik(data, beta))
    g1, g2 = oracle.grad_hess(data, beta)
    for j in range(data.p):
        b1, b2 = brute.grad_hess(data, beta, j)
        assert abs(g1[j] - b1) <= 1e-11 * max(1.0, abs(b1))
        assert abs(g2[j] - b2) <= 1e-11 * max(1.0, abs(b2))


# ------------------------------------------------------------------ finite differences
@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_grad_hess_finite_differences(name, data, opts):
    beta = random_beta(data.p, 0.3, seed=3)
    g1, g2 = oracle.grad_hess(data, beta)
    for j in range(data.p):
        h = 1e-4 * max(1.0, abs(beta[j]))
        bp, bm = beta.copy(), beta.copy()
        bp[j] += h
        bm[j] -= h
        lp, l0, lm = oracle.loglik(data, bp), oracle.loglik(data, beta), oracle.loglik(data, bm)
        fd1 = -(lp - lm) / (2 * h)
        assert abs(fd1 - g1[j]) <= 1e-6 * max(1.0, abs(g1[j])), (j, fd1, g1[j])
        gp, _ = oracle.grad_hess(data, bp, [j])
        gm, _ = oracle.grad_hess(data, bm, [j])
        fd2 = (gp[0] - gm[0]) / (2 * h)
        assert abs(fd2 - g2[j]) <= 1e-6 * max(1.0, abs(g2[j])), (j, fd2, g2[j])


# ------------------------------------------------------------------ closed form
def _three_rows():
    stop = np.array([1, 2, 3]); ev = np.array([1, 1, 1])
    return synth.finalize(stop, ev, None, None, [np.array([0, 2])], [np.array([1.0, 1.0])], 1)


def test_closed_form_three_rows():
    g = _golden_kv("closed_form_three_rows.txt")
    d = _three_rows()
    bh = g["beta_hat"][0]
    assert abs(oracle.loglik(d, np.array([0.0])) - g["loglik_at_zero"][0]) < 1e-15
    assert abs(oracle.loglik(d, np.array([bh])) - g["loglik_at_beta_hat"][0]) < 1e-14
    g1, g2 = oracle.grad_hess(d, np.array([0.0]))
    assert abs(g1[0] - g["g1_at_zero"][0]) < 1e-15 and abs(g2[0] - g["g2_at_zero"][0]) < 1e-15
    g1, g2 = oracle.grad_hess(d, np.array([bh]))
    assert abs(g1[0]) < 1e-15 and abs(g2[0] - g["neg_hessian_at_beta_hat"][0]) < 1e-14
    a1, a2 = oracle.grad_hess(d, np.array([0.0]))
    s, tr = oracle.step(a1[0], a2[0], 0.0, 1.0, synth.PEN_NONE)
    s_, g_ = oracle.step(1 / 6, 17 / 36, 0.0, 1.0, synth.PEN_NONE)
    assert abs(s - g["first_step"][0]) < 1e-15 and abs(s_ - g["first_step"][0]) < 1e-15
    beta, info = oracle.fit(d, synth.CoxOptions(penalty=synth.PEN_NONE, tol=1e-15, max_sweeps=200))
    assert abs(beta[0] - bh) < 1e-12 and info["converged"]


def test_logrank_special_case():
    """At beta = 0 with one binary covariate, g'(0) = -(O - E) and g''(0) is the Breslow
    log-rank variance sum_t d_t (n1/n)(1 - n1/n) -- counted here with integers only."""
    rng = np.random.default_rng(8)
    n = 80
    stop = rng.integers(1, 12, n)
    ev = (rng.random(n) < 0.6).astype(int)
    grp = rng.random(n) < 0.4
    d = synth.finalize(stop, ev, None, None, [np.nonzero(grp)[0]], None, 1)
    x = d.dense_x()[:, 0]
    O = float((x * d.event).sum())
    E = V = 0.0
    for t in np.unique(d.stop[d.event == 1]):
        risk = d.stop >= t
        dt = int(((d.stop == t) & (d.event == 1)).sum())
        nt, n1 = int(risk.sum()), int((risk & (x == 1)).sum())
        E += dt * n1 / nt
        V += dt * (n1 / nt) * (1 - n1 / nt)
    g1, g2 = oracle.grad_hess(d, np.zeros(1))
    assert abs(g1[0] - (-(O - E))) < 1e-12 and abs(g2[0] - V) < 1e-12


# ------------------------------------------------------------------ invariants
def test_stratified_is_sum_of_strata():
    """Eq. strat_l: the stratified partial likelihood is the product over strata."""
    d, _ = synth.stratified_sparse(n=300, p=4, k=6, n_support=2, event_frac=0.3, dens_lo=0.05, dens_hi=0.5,
                                   admin_days=40, seed=21)
    beta = random_beta(d.p, 0.5, seed=4)
    ll = oracle.loglik(d, beta)
    g1, g2 = oracle.grad_hess(d, beta)
    parts_ll, parts_g1, parts_g2 = [], np.zeros(d.p), np.zeros(d.p)
    for kk in np.unique(d.stratum):
        rows = np.nonzero(d.stratum == kk)[0]
        sub = synth.subset_rows(d, rows)
        sub.stratum = None
        parts_ll.append(oracle.loglik(sub, beta))
        a, b = oracle.grad_hess(sub, beta)
        parts_g1 += a
        parts_g2 += b
    assert abs(ll - math.fsum(parts_ll)) <= 1e-12 * abs(ll)
    assert np.allclose(g1, parts_g1, rtol=1e-11, atol=1e-11) and np.allclose(g2, parts_g2, rtol=1e-11, atol=1e-11)


def _split_rows(d, rng):
    """Split every counting-process row with stop - start >= 2 at an interior day, covariates unchanged."""
    n = d.n
    start = d.start if d.start is not None else np.full(n, -1, np.int64)
    keep_rows, new_start, new_stop, new_ev, new_str, src = [], [], [], [], [], []
    for r in range(n):
        s, e = int(start[r]), int(d.stop[r])
        kk = 0 if d.stratum is None else int(d.stratum[r])
        if e - s >= 2 and rng.random() < 0.7:
            c = int(rng.integers(s + 1, e))
            new_start += [s, c]; new_stop += [c, e]; new_ev += [0, int(d.event[r])]; new_str += [kk, kk]; src += [r, r]
        else:
            new_start.append(s); new_stop.append(e); new_ev.append(int(d.event[r])); new_str.append(kk); src.append(r)
    src = np.array(src)
    x = d.dense_x()[src]
    cols = [np.nonzero(x[:, j])[0] for j in range(d.p)]
    vals = [x[c, j] for j, c in enumerate(cols)] if d.val is not None else None
    return synth.finalize(np.array(new_stop), np.array(new_ev), None if d.stratum is None else np.array(new_str),
                          np.array(new_start), cols, vals, d.p)


@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_split_followup_invariant(name, data, opts):
    """§2.2: splitting (start, stop] into pieces with unchanged covariates changes nothing."""
    rng = np.random.default_rng(9)
    sp = _split_rows(data, rng)
    assert sp.n > data.n
    beta = random_beta(data.p, 0.4, seed=5)
    assert abs(oracle.loglik(sp, beta) - oracle.loglik(data, beta)) <= 1e-12 * abs(oracle.loglik(data, beta))
    a1, a2 = oracle.grad_hess(sp, beta)
    b1, b2 = oracle.grad_hess(data, beta)
    assert np.allclose(a1, b1, rtol=1e-11, atol=1e-11) and np.allclose(a2, b2, rtol=1e-11, atol=1e-11)
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-13, max_sweeps=500)
    fa, _ = oracle.fit(sp, o)
    fb, _ = oracle.fit(data, o)
    assert np.allclose(fa, fb, rtol=1e-9, atol=1e-11)


def test_counting_process_with_early_entry_equals_right_censored():
    """With start before every event time the sweep path (R7) must equal the scan path (§2.7)."""
    d, _ = synth.stratified_sparse(n=200, p=4, k=3, n_support=2, event_frac=0.4, dens_lo=0.1, dens_hi=0.5,
                                   admin_days=25, seed=22)
    cp = synth.CoxData(**{**d.__dict__})
    cp.start = np.full(d.n, -1, np.int32)
    beta = random_beta(d.p, 0.5, seed=6)
    assert abs(oracle.loglik(cp, beta) - oracle.loglik(d, beta)) <= 1e-13 * abs(oracle.loglik(d, beta))
    for j in range(d.p):
        a = oracle.risk_sums(cp, beta, j)
        b = oracle.risk_sums(d, beta, j)
        for x, y in zip(a, b):
            assert np.allclose(x, y, rtol=1e-13, atol=0)


def test_augmented_interval_strata_equal_counting_process():
    """§2.2 eq. time_cov_strat_l: covariates piecewise constant on a global grid; the model
    stratified on the K intervals with the augmented X, Y^aug = min(Y, t_k) and
    delta^aug = delta * 1[Y in [t_{k-1}, t_k)] has the same likelihood as the time-varying model."""
    rng = np.random.default_rng(10)
    n, p, grid = 40, 3, [0, 4, 9, 15]       # intervals [0,4), [4,9), [9,15); Y in 1..14
    K = len(grid) - 1
    y = rng.integers(1, 15, n)
    ev = (rng.random(n) < 0.7).astype(int)
    xk = rng.integers(0, 2, (K, n, p)).astype(float)
    # counting-process rows: interval k covers integer times t with t_{k-1} <= t < t_k, i.e.
    # (t_{k-1} - 1, t_k - 1], truncated at Y
    stop_c, start_c, ev_c, xs = [], [], [], []
    for i in range(n):
        for k in range(K):
            s, e = grid[k] - 1, min(grid[k + 1] - 1, int(y[i]))
            if e > s:
                start_c.append(s); stop_c.append(e); ev_c.append(int(ev[i]) if e == y[i] else 0); xs.append(xk[k, i])
    xs = np.array(xs)
    cp = synth.finalize(np.array(stop_c), np.array(ev_c), None, np.array(start_c),
                        [np.nonzero(xs[:, j])[0] for j in range(p)], None, p)
    # augmented stratified form (paper): stratum k holds all n subjects with Y^aug = min(Y, t_k)
    stop_a, ev_a, str_a, xa = [], [], [], []
    for k in range(K):
        for i in range(n):
            stop_a.append(min(int(y[i]), grid[k + 1]))
            ev_a.append(int(ev[i]) if grid[k] <= y[i] < grid[k + 1] else 0)
            str_a.append(k)
            xa.append(xk[k, i])
    xa = np.array(xa)
    aug = synth.finalize(np.array(stop_a), np.array(ev_a), np.array(str_a), None,
                         [np.nonzero(xa[:, j])[0] for j in range(p)], None, p)
    beta = random_beta(p, 0.6, seed=7)
    la, lc = oracle.loglik(aug, beta), oracle.loglik(cp, beta)
    assert abs(la - lc) <= 1e-12 * abs(lc)
    a1, a2 = oracle.grad_hess(aug, beta)
    c1, c2 = oracle.grad_hess(cp, beta)
    assert np.allclose(a1, c1, rtol=1e-11, atol=1e-12) and np.allclose(a2, c2, rtol=1e-11, atol=1e-12)


def test_time_varying_coefficient_split():
    """§2.3: a step-function coefficient at t_s is two time-varying covariates. With equal
    coefficients the likelihood equals the original; with t_s beyond every time the 'after'
    column is zero on every row, so its g' and g'' vanish and the other coefficients fit as before."""
    d, _ = synth.stratified_sparse(n=120, p=3, k=2, n_support=2, event_frac=0.5, dens_lo=0.2, dens_hi=0.6,
                                   admin_days=20, seed=23)
    x = d.dense_x()
    for ts in (8, 10_000):
        rows_s, rows_e, ev_s, st_s, xr = [], [], [], [], []
        for r in range(d.n):
            s0, e0 = -1, int(d.stop[r])
            pieces = [(s0, min(e0, ts - 1), True), (max(s0, ts - 1), e0, False)]
            for a, b, before in pieces:
                if b > a:
                    rows_s.append(a); rows_e.append(b); st_s.append(int(d.stratum[r]))
                    ev_s.append(int(d.event[r]) if b == e0 else 0)
                    xr.append([x[r, 0] if before else 0.0, 0.0 if before else x[r, 0], *x[r, 1:]])
        xr = np.array(xr)
        aug = synth.finalize(np.array(rows_e), np.array(ev_s), np.array(st_s), np.array(rows_s),
                             [np.nonzero(xr[:, j])[0] for j in range(4)], None, 4)
        b = random_beta(3, 0.5, seed=8)
        ba = np.array([b[0], b[0], b[1], b[2]])
        assert abs(oracle.loglik(aug, ba) - oracle.loglik(d, b)) <= 1e-12 * abs(oracle.loglik(d, b))
        if ts > d.stop.max():
            g1, g2 = oracle.grad_hess(aug, ba, [1])
            assert g1[0] == 0.0 and g2[0] == 0.0
            o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-13)
            fa, _ = oracle.fit(aug, o)
            fb, _ = oracle.fit(d, o)
            assert fa[1] == 0.0 and np.allclose(fa[[0, 2, 3]], fb, rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------------ the step rule
def test_step_rule_hand_worked():
    L1, L2, NONE = synth.PEN_L1, synth.PEN_L2, synth.PEN_NONE
    # plain Newton inside the trust region; trust update max(2|s|, tr/2)
    assert oracle.step(0.3, 2.0, 0.0, 1.0, NONE) == (-0.15, 0.5)
    # Newton step clipped by the trust region
    assert oracle.step(-5.0, 1.0, 0.0, 1.0, NONE) == (1.0, 2.0)
    # L2 adds beta/sigma^2 and 1/sigma^2: g' = 0.5 + 1/0.5, g'' = 1 + 1/0.5
    s, t = oracle.step(0.5, 1.0, 1.0, 10.0, L2, l2_var=0.5)
    assert abs(s - (-(0.5 + 2.0) / 3.0)) < 1e-15
    # L1 at 0: both directional derivatives >= 0 -> no move, trust halves
    assert oracle.step(0.4, 1.0, 0.0, 1.0, L1, lam=0.5) == (0.0, 0.5)
    # L1 at 0, g' + gamma < 0 -> move up by -(g'+gamma)/g''
    assert oracle.step(-0.9, 2.0, 0.0, 1.0, L1, lam=0.5) == (0.2, 0.5)
    # L1 at 0, g' - gamma > 0 -> move down by -(g'-gamma)/g''
    assert oracle.step(0.9, 2.0, 0.0, 1.0, L1, lam=0.5) == (-0.2, 0.5)
    # L1 away from 0 uses g' + gamma sgn(beta)
    s, _ = oracle.step(-0.1, 1.0, 0.5, 1.0, L1, lam=0.3)
    assert abs(s - (-0.2)) < 1e-15
    # a step that would cross 0 stops at 0
    assert oracle.step(2.0, 1.0, 0.5, 10.0, L1, lam=0.3)[0] == -0.5
    # unpenalized coordinate under L1 (penalize mask 0) takes the plain Newton step
    assert oracle.step(0.4, 1.0, 0.0, 1.0, L1, lam=0.5, penalized=0)[0] == -0.4
    # g'' <= 0 -> skip
    assert oracle.step(1.0, 0.0, 0.0, 1.0, NONE) == (0.0, 0.5)
    # agreement with the independent restatement in tests/brute.py on random inputs
    rng = np.random.default_rng(3)
    for _ in range(2000):
        args = (rng.normal(), abs(rng.normal()) + 1e-3, rng.choice([0.0, rng.normal()]), abs(rng.normal()) + 0.01)
        pen = int(rng.integers(0, 3))
        lam, var, m = abs(rng.normal()), abs(rng.normal()) + 0.1, int(rng.integers(0, 2))
        a = oracle.step(*args, pen, lam, var, m)
        b = brute.step(*args, pen, lam, var, bool(m))
        assert abs(a[0] - b[0]) <= 1e-14 * max(1, abs(b[0])) and abs(a[1] - b[1]) <= 1e-14 * max(1, b[1])


# ------------------------------------------------------------------ full fits
@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_fit_matches_brute_ccd(name, data, opts):
    o = synth.CoxOptions(penalty=opts.penalty, lam=opts.lam if opts.penalty == 1 else 0.0,
                         l2_var=opts.l2_var, tol=1e-10, max_sweeps=40)
    if o.penalty == synth.PEN_L1:
        o.lam = 0.5
    bo, info = oracle.fit(data, o)
    bb, sweeps, conv = brute.fit(data, o)
    assert info["sweeps"] == sweeps and info["converged"] == conv
    assert np.max(np.abs(bo - bb)) <= 1e-9 * max(np.max(np.abs(bb)), 1e-300) + 1e-14


def test_fit_kkt_conditions():
    d, _ = synth.stratified_sparse(n=400, p=8, k=4, n_support=4, event_frac=0.3, dens_lo=0.05, dens_hi=0.5,
                                   admin_days=60, seed=24)
    for pen, lam, var in ((synth.PEN_L2, 0.0, 0.5), (synth.PEN_L1, 2.0, 1.0)):
        o = synth.CoxOptions(penalty=pen, lam=lam, l2_var=var, tol=1e-15, max_sweeps=3000)
        beta, info = oracle.fit(d, o)
        g1, g2 = oracle.grad_hess(d, beta)
        for j in range(d.p):
            if pen == synth.PEN_L2:
                assert abs(g1[j] + beta[j] / var) < 1e-6
            elif beta[j] != 0.0:
                assert abs(g1[j] + math.copysign(lam, beta[j])) < 1e-6
            else:
                assert abs(g1[j]) <= lam + 1e-9


def test_first_sweep_loglik_monotone_l2():
    """Each CCD sweep with an L2 penalty decreases the penalized objective (convex, trust-region Newton)."""
    d, o = synth.plain_dense(n=200, p=6, seed=31)
    prev = None
    for s in range(1, 8):
        _, info = oracle.fit(d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=0.0, max_sweeps=s))
        if prev is not None:
            assert info["objective"] <= prev + 1e-12
        prev = info["objective"]


# ------------------------------------------------------------------ invariants of eq. strat_l
def _rebuild(d, rows, stop, start, extra_col=None):
    """The rows ``rows`` of d (repeats allowed) with new stop/start days and optionally one more
    column, through the generators' sort and CSC builder."""
    x = d.dense_x()[rows]
    if extra_col is not None:
        x = np.column_stack([x, extra_col])
    p = x.shape[1]
    cols = [np.nonzero(x[:, j])[0] for j in range(p)]
    vals = [x[c, j] for j, c in enumerate(cols)] if (d.val is not None or extra_col is not None) else None
    return synth.finalize(np.asarray(stop), d.event[rows], None if d.stratum is None else d.stratum[rows],
                          None if start is None else np.asarray(start), cols, vals, p)


@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_time_rescaling_invariant(name, data, opts):
    """The partial likelihood sees event times only through their order (risk sets and tie groups):
    stretching every day by 3 changes nothing."""
    rows = np.arange(data.n)
    sc = _rebuild(data, rows, 3 * data.stop.astype(np.int64),
                  None if data.start is None else 3 * data.start.astype(np.int64))
    beta = random_beta(data.p, 0.4, seed=6)
    l0 = oracle.loglik(data, beta)
    assert abs(oracle.loglik(sc, beta) - l0) <= 1e-13 * abs(l0)
    a1, a2 = oracle.grad_hess(sc, beta)
    b1, b2 = oracle.grad_hess(data, beta)
    assert np.allclose(a1, b1, rtol=1e-12, atol=1e-13) and np.allclose(a2, b2, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_row_duplication(name, data, opts):
    """Every row twice: each risk-set sum and each tie group's events double, so
    l2(beta) = 2 l(beta) - 2 D log 2 (D events), and the gradient and curvature double."""
    rows = np.repeat(np.arange(data.n), 2)
    du = _rebuild(data, rows, data.stop[rows], None if data.start is None else data.start[rows])
    beta = random_beta(data.p, 0.4, seed=7)
    D = int(data.event.sum())
    l0 = oracle.loglik(data, beta)
    assert abs(oracle.loglik(du, beta) - (2 * l0 - 2 * D * math.log(2.0))) <= 1e-12 * abs(l0)
    a1, a2 = oracle.grad_hess(du, beta)
    b1, b2 = oracle.grad_hess(data, beta)
    assert np.allclose(a1, 2 * b1, rtol=1e-12, atol=1e-12) and np.allclose(a2, 2 * b2, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name,data,opts", [c for c in tiny_cases() if c[1].stratum is not None])
def test_stratum_constant_column(name, data, opts):
    """A covariate constant within every stratum cancels from every ratio S1/S0 of eq. strat_g:
    its gradient and curvature vanish at any beta, and the fit leaves its coefficient at 0."""
    ks = np.unique(data.stratum)
    level = np.random.default_rng(8).uniform(0.5, 2.0, int(ks.max()) + 1)
    col = level[data.stratum]
    ex = _rebuild(data, np.arange(data.n), data.stop, data.start, extra_col=col)
    beta = np.append(random_beta(data.p, 0.4, seed=9), 0.7)
    g1, g2 = oracle.grad_hess(ex, beta)
    scale = max(1.0, float(np.max(np.abs(g1[:-1]))))
    assert abs(g1[-1]) <= 1e-12 * scale and abs(g2[-1]) <= 1e-12 * max(1.0, float(np.max(g2[:-1])))
    o = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-12, max_sweeps=200)
    b, _ = oracle.fit(ex, o)
    b0, _ = oracle.fit(data, o)
    assert abs(b[-1]) <= 1e-10 and np.allclose(b[:-1], b0, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("name,data,opts", tiny_cases())
def test_time_sample_is_the_fits_first_steps(name, data, opts):
    """The timed CPU baseline (a bounded sample of k coordinate steps from beta = 0) does the fit's
    own work: after k < p steps its coefficients are the first sweep's first k coefficients (the
    cyclic order visits j = 0..k-1 first, and later coordinates have not moved), and after two
    full sweeps they are the two-sweep fit's. Same arithmetic in the same order: bit-exact."""
    o = synth.CoxOptions(penalty=opts.penalty, lam=opts.lam, l2_var=opts.l2_var, tol=0.0, max_sweeps=2)
    b1, _ = oracle.fit(data, synth.CoxOptions(penalty=opts.penalty, lam=opts.lam, l2_var=opts.l2_var, tol=0.0,
                                              max_sweeps=1))
    b2, _ = oracle.fit(data, o)
    k = data.p // 2 + 1
    _, bk = oracle.time_sample(data, o, k, return_beta=True)
    assert np.array_equal(bk[:k], b1[:k]) and not np.any(bk[k:])
    _, bs = oracle.time_sample(data, o, 2 * data.p, return_beta=True)
    assert np.array_equal(bs, b2)
