"""Brute-force Cox quantities written straight from the definitions (paper §2.1-§2.4).

Independent of both the C oracle and the CUDA library: risk sets are formed row by row from
their definition (O(n) per event time), sums use math.fsum. Small inputs only.
"""
from __future__ import annotations

import math

import numpy as np


def _dense(data):
    return data.dense_x()


def groups(data):
    """Tie groups as (stratum id, time, event count), ordered by stratum then time."""
    k = np.zeros(data.n, np.int64) if data.stratum is None else data.stratum.astype(np.int64)
    out = {}
    for r in range(data.n):
        if data.event[r]:
            key = (int(k[r]), int(data.stop[r]))
            out[key] = out.get(key, 0) + 1
    return [(kk, t, d) for (kk, t), d in sorted(out.items())]


def at_risk(data, kk, t):
    """Boolean mask of rows at risk at time t in stratum kk (stop >= t, and start < t)."""
    k = np.zeros(data.n, np.int64) if data.stratum is None else data.stratum.astype(np.int64)
    m = (k == kk) & (data.stop >= t)
    if data.start is not None:
        m &= data.start < t
    return m


def risk_sums(data, beta, j):
    x = _dense(data)
    eta = x @ beta
    e = np.exp(eta)
    S0, S1, S2 = [], [], []
    for kk, t, d in groups(data):
        m = at_risk(data, kk, t)
        S0.append(math.fsum(e[m]))
        if j >= 0:
            S1.append(math.fsum(x[m, j] * e[m]))
            S2.append(math.fsum(x[m, j] ** 2 * e[m]))
        else:
            S1.append(0.0)
            S2.append(0.0)
    return np.array(S0), np.array(S1), np.array(S2)


def risk_count(data):
    return np.array([int(at_risk(data, kk, t).sum()) for kk, t, d in groups(data)], dtype=np.int64)


def loglik(data, beta):
    """Log partial likelihood (eq. strat_l / time_cov_l), summed over event rows."""
    x = _dense(data)
    eta = x @ beta
    e = np.exp(eta)
    k = np.zeros(data.n, np.int64) if data.stratum is None else data.stratum.astype(np.int64)
    terms = []
    for i in range(data.n):
        if data.event[i]:
            m = at_risk(data, int(k[i]), int(data.stop[i]))
            terms.append(eta[i] - math.log(math.fsum(e[m])))
    return math.fsum(terms)


def grad_hess(data, beta, j):
    """g'(beta_j), g''(beta_j) of -loglik (eqs. strat_g, strat_h), over event rows."""
    x = _dense(data)
    eta = x @ beta
    e = np.exp(eta)
    k = np.zeros(data.n, np.int64) if data.stratum is None else data.stratum.astype(np.int64)
    g1, g2 = [], []
    for i in range(data.n):
        if data.event[i]:
            m = at_risk(data, int(k[i]), int(data.stop[i]))
            s0 = math.fsum(e[m])
            s1 = math.fsum(x[m, j] * e[m])
            s2 = math.fsum(x[m, j] ** 2 * e[m])
            g1.append(-x[i, j] + s1 / s0)
            g2.append(s2 / s0 - (s1 / s0) ** 2)
    return math.fsum(g1), math.fsum(g2)


def step(g1, g2, b, tr, penalty, lam=0.0, l2_var=1.0, penalized=True):
    """One coordinate step, restated from §2.4: Newton on the penalized 1-D objective, the
    L1 directional-derivative rule at 0, trust-region clipping, and stop-at-zero for L1."""
    gamma = 0.0
    if penalized and penalty == 2:
        g1, g2 = g1 + b / l2_var, g2 + 1.0 / l2_var
    if penalized and penalty == 1:
        gamma = lam
    if not (g2 > 0) or not math.isfinite(g1):
        s = 0.0
    elif gamma > 0:
        if b == 0.0:
            up, down = g1 + gamma, -g1 + gamma      # directional derivatives along +1 / -1
            if up < 0:
                s = -(g1 + gamma) / g2
            elif down < 0:
                s = -(g1 - gamma) / g2
            else:
                s = 0.0
        else:
            s = -(g1 + math.copysign(gamma, b)) / g2
    else:
        s = -g1 / g2
    s = max(-tr, min(tr, s))
    if gamma > 0 and b != 0.0 and (b + s) * b < 0:
        s = -b
    return s, max(2 * abs(s), tr / 2)


def penalty_value(opts, beta):
    m = np.ones(len(beta), bool) if opts.penalize is None else np.asarray(opts.penalize, bool)
    if opts.penalty == 1:
        return math.fsum(opts.lam * abs(b) for b, mm in zip(beta, m) if mm)
    if opts.penalty == 2:
        return math.fsum(b * b / (2 * opts.l2_var) for b, mm in zip(beta, m) if mm)
    return 0.0


def fit(data, opts, max_sweeps=None):
    """CCD with brute-force derivatives (O(n^2) per coordinate)."""
    p = data.p
    beta = np.zeros(p)
    tr = np.ones(p)
    ms = opts.max_sweeps if max_sweeps is None else max_sweeps
    obj_prev = -loglik(data, beta) + penalty_value(opts, beta)
    sweeps, conv = 0, False
    while sweeps < ms:
        for j in range(p):
            g1, g2 = grad_hess(data, beta, j)
            pen = True if opts.penalize is None else bool(opts.penalize[j])
            s, tr[j] = step(g1, g2, beta[j], tr[j], opts.penalty, opts.lam, opts.l2_var, pen)
            beta[j] += s
        sweeps += 1
        obj = -loglik(data, beta) + penalty_value(opts, beta)
        if abs(obj - obj_prev) <= opts.tol * abs(obj):
            conv = True
            break
        obj_prev = obj
    return beta, sweeps, conv


def loglik_step_coef(data, beta_view, cuts, tvc_cols):
    """Log partial likelihood of a model whose listed coefficients step at the cut days
    (eq. time_coef_l), from the unsplit data: at an event time t in interval k
    (t_k <= t < t_{k+1}), every row's linear predictor uses the interval-k coefficient of each
    listed column. ``beta_view`` is ordered as the split columns (each listed column replaced
    by one coefficient per interval, interval 0 first)."""
    cuts = list(cuts)
    tv = set(int(j) for j in tvc_cols)
    col, c = [], 0
    for j in range(data.p):
        col.append(c)
        c += len(cuts) + 1 if j in tv else 1
    x = _dense(data)
    k = np.zeros(data.n, np.int64) if data.stratum is None else data.stratum.astype(np.int64)
    terms = []
    for i in range(data.n):
        if not data.event[i]:
            continue
        t = int(data.stop[i])
        kk = sum(1 for u in cuts if u <= t)          # interval of t
        b_t = np.array([beta_view[col[j] + (kk if j in tv else 0)] for j in range(data.p)])
        eta = x @ b_t
        m = at_risk(data, int(k[i]), t)
        terms.append(eta[i] - math.log(math.fsum(np.exp(eta[m]))))
    return math.fsum(terms)
