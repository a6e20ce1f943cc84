"""Seeded synthetic survival data shaped like the paper's workloads.

The paper's cohorts (Optum EHR, LEGEND-HTN) are not available, so every input is drawn
here from a stated recipe with NumPy's PCG64 generator. This module only *draws data*:
it evaluates no partial likelihood, gradient, Hessian or coordinate step. Both the CUDA
path and the CPU oracle receive its arrays as plain inputs; neither imports the other.

Every data set is returned in the layout the library expects (paper §2.7: observations of
a stratum are concatenated and ordered by time): rows sorted by (stratum ascending, stop
ascending, original index), and X as CSC over the sorted rows with row indices ascending
within each column.

Recipes (one function each):

* ``plain_dense``       — N=1e3, p=10 dense N(0,1) covariates, exponential event times
                          rounded up to integer days (heavy ties), ~30 % uniform censoring.
* ``stratified_sparse`` — N=2e6, p=2000 binary columns with log-uniform density, Zipf(1.1)
                          strata sizes, Weibull(1.5) times, ~5 % events (paper §3.1 shape).
* ``time_varying``      — 1e6 subjects split into (start, stop] counting-process rows with
                          per-interval covariates, piecewise-exponential events (§2.2 shape).
* ``batch_views`` / ``serving_stream`` — many uneven fits (cross-validation folds x
                          penalty grid x outcomes) and a Poisson request stream.

All sizes are parameters so the tests can draw small instances of the same recipe.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 2310162380

PEN_NONE, PEN_L1, PEN_L2 = 0, 1, 2


@dataclasses.dataclass
class CoxData:
    """Time-sorted survival data with a CSC design matrix (host arrays)."""

    stop: np.ndarray                      # int32[n], integer days
    event: np.ndarray                     # uint8[n], 1 = event at ``stop``
    col_ptr: np.ndarray                   # int64[p+1]
    row_idx: np.ndarray                   # int32[nnz]
    p: int
    start: Optional[np.ndarray] = None    # int32[n] or None (no counting-process rows)
    stratum: Optional[np.ndarray] = None  # int32[n] or None (one stratum)
    val: Optional[np.ndarray] = None      # float64[nnz] or None (binary X)
    beta_true: Optional[np.ndarray] = None
    recipe: str = ""

    @property
    def n(self) -> int:
        return int(self.stop.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.row_idx.shape[0])

    def dense_x(self) -> np.ndarray:
        """Dense float64 copy of X (small inputs only)."""
        x = np.zeros((self.n, self.p))
        for j in range(self.p):
            a, b = self.col_ptr[j], self.col_ptr[j + 1]
            x[self.row_idx[a:b], j] = 1.0 if self.val is None else self.val[a:b]
        return x


@dataclasses.dataclass
class CoxOptions:
    penalty: int = PEN_NONE
    lam: float = 0.0          # L1 weight gamma (paper §2.1 penalty)
    l2_var: float = 1.0       # Gaussian-prior variance sigma^2 for L2
    penalize: Optional[np.ndarray] = None  # uint8[p]; None = all coordinates penalized
    tol: float = 1e-8
    max_sweeps: int = 1000


def _sizes_zipf(n: int, k: int, s: float = 1.1) -> np.ndarray:
    w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    exact = w / w.sum() * n
    sizes = np.floor(exact).astype(np.int64)
    rem = n - int(sizes.sum())
    order = np.argsort(-(exact - sizes), kind="stable")
    sizes[order[:rem]] += 1
    return sizes


def _bisect(f, lo: float, hi: float, target: float, iters: int = 80, increasing: bool = True) -> float:
    """Find x in [lo, hi] with f(x) ~= target for a monotone f (log-scale bisection)."""
    a, b = math.log(lo), math.log(hi)
    for _ in range(iters):
        m = 0.5 * (a + b)
        v = f(math.exp(m))
        if (v < target) == increasing:
            a = m
        else:
            b = m
    return math.exp(0.5 * (a + b))


def finalize(stop, event, stratum, start, cols_rows, cols_vals, p, beta_true=None, recipe=""):
    """Sort rows by (stratum, stop, original index) and build the CSC over sorted rows.

    ``cols_rows[j]`` holds the ORIGINAL row ids of column j's nonzeros (any order) and
    ``cols_vals[j]`` their values (or ``cols_vals`` is None for a binary X).
    """
    n = int(stop.shape[0])
    idx = np.arange(n, dtype=np.int64)
    keys = (idx, stop) if stratum is None else (idx, stop, stratum)
    order = np.lexsort(keys)
    newpos = np.empty(n, dtype=np.int64)
    newpos[order] = idx
    lens = np.array([len(r) for r in cols_rows], dtype=np.int64)
    col_ptr = np.zeros(p + 1, dtype=np.int64)
    np.cumsum(lens, out=col_ptr[1:])
    if lens.sum() > 0:
        allrows = np.concatenate([np.asarray(r, dtype=np.int64) for r in cols_rows])
    else:
        allrows = np.zeros(0, dtype=np.int64)
    colid = np.repeat(np.arange(p, dtype=np.int64), lens)
    key = colid * n + newpos[allrows]
    perm = np.argsort(key, kind="stable")
    row_idx = (key[perm] - colid[perm] * n).astype(np.int32)
    val = None
    if cols_vals is not None:
        allv = np.concatenate([np.asarray(v, dtype=np.float64) for v in cols_vals]) if lens.sum() else np.zeros(0)
        val = np.ascontiguousarray(allv[perm])
    return CoxData(
        stop=np.ascontiguousarray(stop[order].astype(np.int32)),
        event=np.ascontiguousarray(event[order].astype(np.uint8)),
        stratum=None if stratum is None else np.ascontiguousarray(stratum[order].astype(np.int32)),
        start=None if start is None else np.ascontiguousarray(start[order].astype(np.int32)),
        col_ptr=col_ptr, row_idx=np.ascontiguousarray(row_idx), val=val, p=p,
        beta_true=beta_true, recipe=recipe)


def plain_dense(n: int = 1000, p: int = 10, censor_frac: float = 0.30, seed: int = SEED_BASE + 1):
    """Unstratified Cox data with dense N(0,1) covariates and heavy Breslow ties.

    beta ~ N(0, 0.5^2); T ~ Exponential(rate exp(x'beta)); C ~ U(0, c) with c chosen by
    bisection so that ~``censor_frac`` of the rows are censored; Y = ceil(min(T, C)) days.
    Options: L2 with prior variance 1, relative objective tolerance 1e-8.
    """
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, p))
    beta = rng.normal(0.0, 0.5, p)
    rate = np.exp(x @ beta)
    t = rng.exponential(1.0, n) / rate
    u = rng.random(n)
    c = _bisect(lambda cc: float(np.mean(u * cc < t)), 1e-4, 1e4, censor_frac, increasing=False)
    cens = u * c
    y = np.maximum(np.ceil(np.minimum(t, cens)), 1).astype(np.int64)
    ev = (t <= cens).astype(np.uint8)
    cols_rows = [np.arange(n)] * p
    cols_vals = [x[:, j] for j in range(p)]
    data = finalize(y, ev, None, None, cols_rows, cols_vals, p, beta, "plain_dense")
    return data, CoxOptions(penalty=PEN_L2, l2_var=1.0, tol=1e-8)


def stratified_sparse(n: int = 2_000_000, p: int = 2000, k: int = 100, n_support: int = 50,
                      event_frac: float = 0.05, admin_days: int = 3650, shape: float = 1.5,
                      dens_lo: float = 1e-4, dens_hi: float = 5e-2, lam_per_n: float = 1e-3,
                      seed: int = SEED_BASE + 2):
    """Large stratified sparse binary fit (paper §3.1 synthetic study shape).

    Strata sizes proportional to k^-1.1 (rounded to sum to n). Column j is Bernoulli with
    density log-uniform in [dens_lo, dens_hi]. ``n_support`` coefficients ~ N(0, 0.3^2),
    the rest 0. T = (-ln U / (h exp(eta)))^(1/shape) (Weibull), administrative censoring at
    ``admin_days`` with h chosen by bisection for ~``event_frac`` events; Y = ceil(min(T, admin)).
    Options: L1 with gamma = lam_per_n * n.
    """
    rng = np.random.default_rng(seed)
    k = max(1, min(k, n))
    sizes = _sizes_zipf(n, k)
    stratum = np.repeat(np.arange(k, dtype=np.int64), sizes)
    dens = np.exp(rng.uniform(math.log(dens_lo), math.log(dens_hi), p))
    cols = []
    for j in range(p):
        m = int(rng.binomial(n, dens[j]))
        cols.append(np.sort(rng.choice(n, size=m, replace=False)))
    beta = np.zeros(p)
    sup = rng.choice(p, size=min(n_support, p), replace=False)
    beta[sup] = rng.normal(0.0, 0.3, len(sup))
    eta = np.zeros(n)
    for j in sup:
        eta[cols[j]] += beta[j]
    u = rng.random(n)
    base = -np.log(u) / np.exp(eta)
    h = _bisect(lambda hh: float(np.mean((base / hh) ** (1.0 / shape) <= admin_days)), 1e-12, 1e3,
                event_frac, increasing=True)
    t = (base / h) ** (1.0 / shape)
    ev = (t <= admin_days).astype(np.uint8)
    y = np.maximum(np.ceil(np.minimum(t, admin_days)), 1).astype(np.int64)
    data = finalize(y, ev, stratum, None, cols, None, p, beta, "stratified_sparse")
    return data, CoxOptions(penalty=PEN_L1, lam=lam_per_n * n, tol=1e-8)


def time_varying(n_subj: int = 1_000_000, p: int = 5000, k: int = 20, density: float = 1e-3,
                 event_frac: float = 0.10, n_support: int = 50, max_intervals: int = 20,
                 l2_var: float = 0.1, seed: int = SEED_BASE + 3):
    """Counting-process (start, stop] rows with per-interval covariates (paper §2.2 shape).

    Follow-up F ~ U{30..3650} days; m = min(Poisson(2)+1, max_intervals) intervals cut at
    m-1 uniform days in [1, F-1] (duplicate cut days merge, so a few subjects get fewer
    rows). Every row draws its own binary covariates with ``density``. Subject hazard is
    piecewise constant, h * exp(x_row'beta) on each row's interval, with h chosen by
    bisection for ~``event_frac`` subjects with an event; the event row is cut at
    ceil(event time) and later rows are dropped. Strata: uniform over k. Options: L2, variance ``l2_var``.
    """
    rng = np.random.default_rng(seed)
    fu = rng.integers(30, 3651, n_subj)
    m = np.minimum(rng.poisson(2.0, n_subj) + 1, max_intervals)
    ncut = m - 1
    subj_of_cut = np.repeat(np.arange(n_subj), ncut)
    cut_day = 1 + np.floor(rng.random(subj_of_cut.shape[0]) * (fu[subj_of_cut] - 1)).astype(np.int64)
    o = np.lexsort((cut_day, subj_of_cut))
    subj_of_cut, cut_day = subj_of_cut[o], cut_day[o]
    keep = np.ones(len(cut_day), dtype=bool)
    keep[1:] = (subj_of_cut[1:] != subj_of_cut[:-1]) | (cut_day[1:] != cut_day[:-1])
    subj_of_cut, cut_day = subj_of_cut[keep], cut_day[keep]
    ncut = np.bincount(subj_of_cut, minlength=n_subj)
    nrow = ncut + 1
    r_total = int(nrow.sum())
    subj = np.repeat(np.arange(n_subj), nrow)
    first = np.zeros(n_subj + 1, dtype=np.int64)
    np.cumsum(nrow, out=first[1:])
    # stops: the cut days then F; starts: 0 then the cut days
    stop = np.empty(r_total, dtype=np.int64)
    start = np.empty(r_total, dtype=np.int64)
    is_last = np.zeros(r_total, dtype=bool)
    is_last[first[1:] - 1] = True
    is_first = np.zeros(r_total, dtype=bool)
    is_first[first[:-1]] = True
    stop[~is_last] = cut_day
    stop[is_last] = fu
    start[is_first] = 0
    start[~is_first] = cut_day
    cols = []
    for j in range(p):
        mm = int(rng.binomial(r_total, density))
        cols.append(np.sort(rng.choice(r_total, size=mm, replace=False)))
    beta = np.zeros(p)
    sup = rng.choice(p, size=min(n_support, p), replace=False)
    beta[sup] = rng.normal(0.0, 0.3, len(sup))
    eta = np.zeros(r_total)
    for j in sup:
        eta[cols[j]] += beta[j]
    w = np.exp(eta) * (stop - start)           # cumulative hazard per row, per unit h
    cumw = np.cumsum(w)
    subj_w = np.add.reduceat(w, first[:-1])
    e_draw = rng.exponential(1.0, n_subj)
    h = _bisect(lambda hh: float(np.mean(e_draw < hh * subj_w)), 1e-12, 1e3, event_frac, increasing=True)
    # locate the event row: first row whose cumulative (within subject) hazard exceeds E
    before = cumw - w                          # global cumulative before row
    subj_base = before[first[:-1]]             # global cumulative before subject's first row
    target = subj_base + e_draw / h            # global cumulative at the event
    has_ev = e_draw < h * subj_w
    ev_row = np.searchsorted(cumw, target, side="left")
    ev_row = np.where(has_ev, np.minimum(ev_row, first[1:] - 1), -1)
    keep_row = np.ones(r_total, dtype=bool)
    event = np.zeros(r_total, dtype=np.uint8)
    sel = np.nonzero(has_ev)[0]
    er = ev_row[sel]
    t_ev = start[er] + (target[sel] - before[er]) / (h * np.exp(eta[er]))
    new_stop = np.minimum(np.maximum(np.ceil(t_ev), start[er] + 1), stop[er]).astype(np.int64)
    stop[er] = new_stop
    event[er] = 1
    # drop rows after the event row
    last_keep = np.where(has_ev, ev_row, first[1:] - 1)
    pos_in = np.arange(r_total) - first[subj]
    keep_row = pos_in <= (last_keep[subj] - first[subj])
    old_to_new = np.full(r_total, -1, dtype=np.int64)
    old_to_new[keep_row] = np.arange(int(keep_row.sum()))
    cols = [old_to_new[c[keep_row[c]]] for c in cols]
    stratum_subj = rng.integers(0, k, n_subj)
    data = finalize(stop[keep_row], event[keep_row], stratum_subj[subj[keep_row]], start[keep_row],
                    cols, None, p, beta, "time_varying")
    return data, CoxOptions(penalty=PEN_L2, l2_var=l2_var, tol=1e-8)


def synthetic_e1(n: int = 1_000_000, p: int = 2000, k: int = 50_000, density: float = 0.05, censor_frac: float = 0.3,
                 seed: int = SEED_BASE + 8):
    """The paper's synthetic experiment (§3.1): binary X with 5 % of the entries set to 1
    uniformly, beta_j ~ N(0, 1) with 80 % of the coefficients set to 0, equal-sized strata
    (rows i.i.d., so stratum = row block), L1 with gamma = sqrt(2). The paper does not state how
    event times are drawn; here T ~ Exp(exp(x'beta)) with independent uniform censoring tuned to
    ``censor_frac``, Y = ceil(100 * min(T, C)) (times on a 1/100 grid)."""
    rng = np.random.default_rng(seed)
    k = max(1, min(k, n))
    cols = []
    for j in range(p):
        m = int(rng.binomial(n, density))
        cols.append(np.sort(rng.choice(n, size=m, replace=False)))
    beta = rng.normal(0.0, 1.0, p) * (rng.random(p) < 0.2)
    eta = np.zeros(n)
    for j in np.flatnonzero(beta):
        eta[cols[j]] += beta[j]
    t = rng.exponential(1.0, n) / np.exp(eta)
    u = rng.random(n)
    c = _bisect(lambda cc: float(np.mean(u * cc < t)), 1e-12, 1e12, censor_frac, iters=120, increasing=False)
    cens = u * c
    ev = (t <= cens).astype(np.uint8)
    scale = 100.0 / float(np.median(np.minimum(t, cens)))
    y = np.maximum(np.ceil(scale * np.minimum(t, cens)), 1).astype(np.int64)
    y = np.minimum(y, 2**31 - 1)
    stratum = (np.arange(n, dtype=np.int64) * k) // n
    data = finalize(y, ev, stratum, None, cols, None, p, beta, "synthetic_e1")
    return data, CoxOptions(penalty=PEN_L1, lam=math.sqrt(2.0), tol=1e-8)


def subset_rows(data: CoxData, rows: np.ndarray) -> CoxData:
    """Restrict a data set to ``rows`` (sorted row ids); keeps the sort order."""
    rows = np.asarray(rows, dtype=np.int64)
    remap = np.full(data.n, -1, dtype=np.int64)
    remap[rows] = np.arange(len(rows))
    cols_rows, cols_vals = [], [] if data.val is not None else None
    for j in range(data.p):
        a, b = data.col_ptr[j], data.col_ptr[j + 1]
        r = remap[data.row_idx[a:b]]
        keep = r >= 0
        cols_rows.append(r[keep])
        if cols_vals is not None:
            cols_vals.append(data.val[a:b][keep])
    return finalize(data.stop[rows], data.event[rows],
                    None if data.stratum is None else data.stratum[rows],
                    None if data.start is None else data.start[rows],
                    cols_rows, cols_vals, data.p, data.beta_true, data.recipe + "/subset")


def _subset_shared(col_ptr, row_idx, rows, n_total):
    """Columns of a shared binary CSC restricted to ``rows`` (original ids), as per-column lists
    of positions within ``rows``."""
    remap = np.full(n_total, -1, dtype=np.int64)
    remap[rows] = np.arange(len(rows))
    r = remap[row_idx]
    keep = r >= 0
    cnt = np.add.reduceat(keep.astype(np.int64), col_ptr[:-1]) if len(row_idx) else np.zeros(len(col_ptr) - 1, np.int64)
    cnt[np.diff(col_ptr) == 0] = 0
    kept = r[keep]
    out, o = [], 0
    for c in cnt:
        out.append(kept[o:o + c])
        o += c
    return out


def batch_views(n_total: int = 1_000_000, p: int = 1000, density: float = 1e-2, n_outcomes: int = 4,
                n_folds: int = 4, n_lambdas: int = 16, n_lo: float = 1e4, n_hi: float = 1e6,
                max_strata: int = 50, event_frac: float = 0.05, seed: int = SEED_BASE + 4):
    """Many uneven fits over one shared sparse X (cross-validation folds x penalty grid x outcomes).

    One binary X of ``n_total`` rows x ``p`` columns (density ``density``). Each outcome draws
    its own Weibull(1.5) event times (20 nonzero coefficients ~ N(0, 0.3^2), administrative
    censoring at 3650 days, ~``event_frac`` events). For every (outcome, fold) pair a training
    set of N ~ logU[n_lo, n_hi] rows is sampled from X, with K ~ U{1..max_strata} strata; each
    training set is fitted at ``n_lambdas`` L1 weights log-spaced over [1e-4, 1e-1] * N.
    Returns a list of (CoxData, [CoxOptions per lambda]) -- one entry per training set.
    """
    rng = np.random.default_rng(seed)
    cols = [np.sort(rng.choice(n_total, size=int(rng.binomial(n_total, density)), replace=False)) for _ in range(p)]
    col_ptr = np.zeros(p + 1, np.int64)
    np.cumsum([len(c) for c in cols], out=col_ptr[1:])
    row_idx = np.concatenate(cols).astype(np.int64)
    sets = []
    for o in range(n_outcomes):
        beta = np.zeros(p)
        sup = rng.choice(p, 20, replace=False)
        beta[sup] = rng.normal(0, 0.3, 20)
        eta = np.zeros(n_total)
        for j in sup:
            eta[cols[j]] += beta[j]
        base = -np.log(rng.random(n_total)) / np.exp(eta)
        h = _bisect(lambda hh: float(np.mean((base / hh) ** (1 / 1.5) <= 3650)), 1e-12, 1e3, event_frac)
        t = (base / h) ** (1 / 1.5)
        ev = (t <= 3650).astype(np.uint8)
        y = np.maximum(np.ceil(np.minimum(t, 3650)), 1).astype(np.int64)
        for f in range(n_folds):
            n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
            rows = np.sort(rng.choice(n_total, size=n, replace=False))
            k = int(rng.integers(1, max_strata + 1))
            stratum = rng.integers(0, k, n)
            sub = _subset_shared(col_ptr, row_idx, rows, n_total)
            data = finalize(y[rows], ev[rows], stratum, None, sub, None, p, beta, f"batch_view o{o} f{f}")
            lams = np.exp(np.linspace(math.log(1e-4), math.log(1e-1), n_lambdas)) * n
            sets.append((data, [CoxOptions(penalty=PEN_L1, lam=float(l), tol=1e-8) for l in lams]))
    return sets


@dataclasses.dataclass
class Request:
    """One fit request of the serving stream."""
    arrival_s: float
    n_subj: int
    p: int
    density: float
    k: int
    counting: bool
    penalty: int
    seed: int


def serving_stream(rate: float = 20.0, duration_s: float = 120.0, n_lo: float = 1e4, n_hi: float = 1e7,
                   p_lo: float = 100, p_hi: float = 2e4, d_lo: float = 1e-4, d_hi: float = 1e-2,
                   k_max: int = 200, seed: int = SEED_BASE + 5):
    """Poisson request arrivals (mean ``rate`` per second over ``duration_s``). Each request
    draws rows ~ logU[n_lo, n_hi], p ~ logU[p_lo, p_hi], density ~ logU[d_lo, d_hi],
    K ~ U{1..k_max}, counting-process rows with probability 1/2 and L1 or L2 with probability
    1/2 each, plus its own data seed. ``request_data`` materializes a request."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        lu = lambda a, b: math.exp(rng.uniform(math.log(a), math.log(b)))
        out.append(Request(t, int(lu(n_lo, n_hi)), int(lu(p_lo, p_hi)), lu(d_lo, d_hi), int(rng.integers(1, k_max + 1)),
                           bool(rng.random() < 0.5), PEN_L1 if rng.random() < 0.5 else PEN_L2,
                           int(rng.integers(0, 2**31 - 1))))
    return out


def request_data(req: Request, max_rows: Optional[int] = None):
    """Data and options of one serving request (counting-process requests use ``time_varying``
    with n_subj / 3 subjects so that the row count is comparable)."""
    n = req.n_subj if max_rows is None else min(req.n_subj, max_rows)
    if req.counting:
        data, opts = time_varying(n_subj=max(10, n // 3), p=req.p, k=req.k, density=req.density,
                                  n_support=min(20, req.p), seed=req.seed)
    else:
        data, opts = stratified_sparse(n=n, p=req.p, k=min(req.k, n), n_support=min(20, req.p),
                                       dens_lo=req.density, dens_hi=req.density * 1.0001, seed=req.seed)
    if req.penalty == PEN_L1:
        opts = CoxOptions(penalty=PEN_L1, lam=1e-4 * data.n, tol=1e-8)
    else:
        opts = CoxOptions(penalty=PEN_L2, l2_var=1.0, tol=1e-8)
    return data, opts
