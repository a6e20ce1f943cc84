"""The seeded input generators follow their stated recipes (CPU, small sizes).

The benchmark and parity workloads are synthetic stand-ins for the paper's cohorts; these tests
check that each generator produces what its recipe says (strata sizes, sort order, CSC layout,
column densities, event or censoring fractions, coefficient support, options), and that a seed
fixes the data.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2310_16238_gb300 import synth


def _check_layout(d: synth.CoxData):
    n = d.n
    assert d.col_ptr.shape == (d.p + 1,) and d.col_ptr[0] == 0 and d.col_ptr[-1] == d.nnz
    assert np.all(np.diff(d.col_ptr) >= 0)
    assert d.nnz == 0 or (d.row_idx.min() >= 0 and d.row_idx.max() < n)
    for j in range(d.p):   # rows ascending and distinct within a column
        r = d.row_idx[d.col_ptr[j]:d.col_ptr[j + 1]]
        assert np.all(np.diff(r) > 0)
    s = np.zeros(n, np.int64) if d.stratum is None else d.stratum.astype(np.int64)
    key = s * (int(d.stop.max()) + 1) + d.stop
    assert np.all(np.diff(key) >= 0), "rows sorted by (stratum, stop)"
    assert set(np.unique(d.event)) <= {0, 1}
    if d.start is not None:
        assert np.all(d.start < d.stop)


def _densities(d):
    return np.diff(d.col_ptr) / d.n


def _logu_mean_sd(lo, hi):
    m = (hi - lo) / math.log(hi / lo)
    m2 = (hi * hi - lo * lo) / (2.0 * math.log(hi / lo))
    return m, math.sqrt(m2 - m * m)


def test_seed_fixes_the_data():
    a, _ = synth.stratified_sparse(n=5000, p=40, k=5)
    b, _ = synth.stratified_sparse(n=5000, p=40, k=5)
    c, _ = synth.stratified_sparse(n=5000, p=40, k=5, seed=synth.SEED_BASE + 99)
    for f in ("stop", "event", "stratum", "col_ptr", "row_idx"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not (np.array_equal(a.stop, c.stop) and np.array_equal(a.row_idx, c.row_idx))


def test_stratified_sparse_recipe():
    n, p, k = 40_000, 300, 20
    d, o = synth.stratified_sparse(n=n, p=p, k=k)
    _check_layout(d)
    sizes = np.bincount(d.stratum, minlength=k)
    assert sizes.sum() == n and np.array_equal(sizes, synth._sizes_zipf(n, k))
    w = np.arange(1, k + 1) ** -1.1
    assert np.all(np.abs(sizes - w / w.sum() * n) < 1.0)          # proportional to k^-1.1, rounded
    assert d.stop.min() >= 1 and d.stop.max() <= 3650
    assert abs(d.event.mean() - 0.05) < 0.005                     # ~5 % events
    assert np.all(d.stop[d.event == 0] == 3650)                   # administrative censoring only
    m, sd = _logu_mean_sd(1e-4, 5e-2)
    dens = _densities(d)
    assert abs(dens.mean() - m) < 4 * sd / math.sqrt(p) and dens.max() < 0.06
    assert np.count_nonzero(d.beta_true) == 50
    assert o.penalty == synth.PEN_L1 and o.lam == pytest.approx(1e-3 * n) and o.tol == 1e-8


def test_time_varying_recipe():
    n_subj, p, k = 5000, 60, 5
    d, o = synth.time_varying(n_subj=n_subj, p=p, k=k, density=0.01)
    _check_layout(d)
    assert d.start is not None and d.start.min() >= 0 and d.stop.max() <= 3650
    assert n_subj <= d.n <= 20 * n_subj                          # 1 to 20 rows per subject
    assert 1.5 < d.n / n_subj < 3.5                              # mean Poisson(2) + 1 rows, shortened by events
    assert abs(d.event.sum() / n_subj - 0.10) < 0.02              # ~10 % of subjects with an event
    assert d.stratum.min() >= 0 and d.stratum.max() < k
    assert abs(_densities(d).mean() - 0.01) < 0.002
    assert o.penalty == synth.PEN_L2 and o.l2_var == 0.1


def test_synthetic_e1_recipe():
    """The paper's §3.1 design: 5 % binary X, 20 % of beta nonzero N(0, 1), equal strata,
    L1 gamma = sqrt(2)."""
    n, p, k = 20_000, 500, 50
    d, o = synth.synthetic_e1(n=n, p=p, k=k)
    _check_layout(d)
    assert np.array_equal(np.bincount(d.stratum, minlength=k), np.full(k, n // k))
    assert abs(_densities(d).mean() - 0.05) < 0.002
    nz = np.count_nonzero(d.beta_true) / p
    assert abs(nz - 0.2) < 0.06
    assert abs(np.std(d.beta_true[d.beta_true != 0]) - 1.0) < 0.2
    assert abs((1 - d.event.mean()) - 0.3) < 0.02                 # ~30 % censored
    assert o.penalty == synth.PEN_L1 and o.lam == pytest.approx(math.sqrt(2.0))


def test_batch_views_recipe():
    """Uneven training sets over one shared X: outcomes x folds sets, each with its penalty grid."""
    n_total, p = 50_000, 80
    sets = synth.batch_views(n_total=n_total, p=p, density=0.02, n_outcomes=2, n_folds=3, n_lambdas=4,
                             n_lo=2e3, n_hi=2e4, max_strata=7)
    assert len(sets) == 6 and all(len(opts) == 4 for _, opts in sets)
    for d, opts in sets:
        _check_layout(d)
        assert 2e3 - 1 <= d.n <= 2e4 + 1 and d.stratum.max() < 7
        assert abs(_densities(d).mean() - 0.02) < 0.004
        lams = np.array([o.lam for o in opts])
        assert lams[0] == pytest.approx(1e-4 * d.n) and lams[-1] == pytest.approx(1e-1 * d.n)
        assert np.allclose(np.diff(np.log(lams)), np.log(1e3) / 3)
        assert np.count_nonzero(d.beta_true) == 20
    # sets of one outcome share its coefficients; the two outcomes differ
    assert np.array_equal(sets[0][0].beta_true, sets[2][0].beta_true)
    assert not np.array_equal(sets[0][0].beta_true, sets[3][0].beta_true)


def test_serving_stream_recipe():
    reqs = synth.serving_stream(rate=20.0, duration_s=200.0)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] <= 200.0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 20.0) < 0.005                    # Poisson arrivals at 20 per second
    assert abs(len(reqs) - 4000) < 4 * math.sqrt(4000)
    n = np.array([r.n_subj for r in reqs], float)
    assert n.min() >= 1e4 - 1 and n.max() <= 1e7
    assert abs(np.log(n).mean() - 0.5 * (math.log(1e4) + math.log(1e7))) < 0.15   # log-uniform rows
    assert abs(np.mean([r.counting for r in reqs]) - 0.5) < 0.04
    assert abs(np.mean([r.penalty == synth.PEN_L1 for r in reqs]) - 0.5) < 0.04
    assert min(r.k for r in reqs) >= 1 and max(r.k for r in reqs) <= 200


def test_device_generators_follow_the_recipes():
    """The torch generators used for serving requests too large for NumPy (run here on CPU
    tensors): sorted rows, a valid CSC, the recipe's densities and event fractions."""
    torch = pytest.importorskip("torch")
    from paper_2310_16238_gb300 import synth_device as sd
    for d, dens, ev in ((sd.stratified_sparse(40000, 40, 9, 0.01, 5, "cpu"), 0.01, 0.05),
                        (sd.time_varying(12000, 30, 4, 0.01, 6, "cpu"), 0.01, None)):
        host = synth.CoxData(stop=d.stop.numpy(), event=d.event.numpy(), col_ptr=d.col_ptr.numpy(),
                             row_idx=d.row_idx.numpy(), p=d.p, stratum=d.stratum.numpy(),
                             start=None if d.start is None else d.start.numpy())
        _check_layout(host)
        assert abs(np.diff(host.col_ptr).mean() / host.n - dens) < 0.1 * dens
        if ev is not None:
            assert abs(host.event.mean() - ev) < 0.2 * ev
        else:
            assert np.all(host.start < host.stop)
