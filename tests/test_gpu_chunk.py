"""The FP32C streaming kernel with chunks of several tiles, against the oracle.

The kernel streams each fit as chunks of consecutive 4,096-position tiles, carrying sums from tile
to tile inside a chunk and through one look-back between chunks; tie groups whose risk set runs
past their chunk wait for its carry. On small data the library's own plan gives every chunk one
tile, so these tests force 1 to 7 tiles per chunk (cox_debug_set_chunk_tiles): fits, gradients and
log-likelihoods must match the oracle at the FP32C tolerances (beta 1e-5 relative to max |beta|,
log-likelihood 1e-7 of its scale), whatever the chunk length -- on strata and tie groups that span
chunks, counting-process sequences, head-capped tiles and a batch of uneven fits.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import synth
from tests.cases import random_beta

pytestmark = pytest.mark.gpu
cox = pytest.importorskip("paper_2310_16238_gb300.cox")

CHUNK_TILES = (1, 2, 3, 7)


def _rel_beta(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)) if len(b) else 0.0


def _ll_scale(data, beta, ll):
    return max(abs(ll), float(np.sum(data.event)))


@pytest.fixture
def chunk_tiles(request):
    cox.cox_debug_set_chunk_tiles(request.param)
    yield request.param
    cox.cox_debug_set_chunk_tiles(0)


def _cases():
    out = []
    # one stratum over ~12 tiles: every chunk's groups wait for the next chunk's carry
    d, o = synth.stratified_sparse(n=50000, p=12, k=1, n_support=5, event_frac=0.2, dens_lo=0.005, dens_hi=0.2,
                                   admin_days=2000, lam_per_n=1e-4, seed=61)
    out.append(("one_stratum_l1", d, o))
    # many strata (ends inside and on the edges of tiles and chunks), L2
    d, _ = synth.stratified_sparse(n=60000, p=10, k=40, n_support=5, event_frac=0.1, dens_lo=0.005, dens_hi=0.3,
                                   admin_days=400, seed=62)
    out.append(("many_strata_l2", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=0.5, tol=1e-10)))
    # counting process: exits carry -exp(eta)
    d, o = synth.time_varying(n_subj=12000, p=10, k=3, density=0.05, event_frac=0.3, n_support=5, seed=63)
    out.append(("counting_l2", d, o))
    # more tie groups than a tile holds: shortened, head-capped tiles inside chunks
    rng = np.random.default_rng(64)
    n = 40000
    d = synth.finalize(np.arange(n) + 1, np.ones(n, int), rng.integers(0, 2, n), None,
                       [np.nonzero(rng.random(n) < 0.1)[0] for _ in range(4)], None, 4)
    out.append(("head_capped", d, synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-10)))
    # valued X
    d, o = synth.plain_dense(n=30000, p=6, seed=65)
    out.append(("dense_valued", d, o))
    return out


CASES = _cases()
_ORACLE = {}


def _oracle_fit(name, data, opts, max_sweeps=None):
    """The oracle's fit, cached across chunk lengths (it does not depend on them)."""
    key = (name, max_sweeps)
    if key not in _ORACLE:
        _ORACLE[key] = oracle.fit(data, opts, max_sweeps=max_sweeps)
    return _ORACLE[key]


@pytest.mark.parametrize("chunk_tiles", CHUNK_TILES, indirect=True)
@pytest.mark.parametrize("name,data,opts", CASES, ids=[c[0] for c in CASES])
def test_fp32c_fit_with_multi_tile_chunks(name, data, opts, chunk_tiles):
    with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) as h:
        beta, info = h.fit()
    ob, oinfo = _oracle_fit(name, data, opts, info["sweeps"])
    ob2, oinfo2 = _oracle_fit(name, data, opts)
    err = min(_rel_beta(beta, ob), _rel_beta(beta, ob2))
    assert err <= 1e-5, (err, chunk_tiles)
    assert abs(info["loglik"] - oinfo2["loglik"]) <= 1e-7 * _ll_scale(data, ob2, oinfo2["loglik"])


@pytest.mark.parametrize("chunk_tiles", CHUNK_TILES, indirect=True)
@pytest.mark.parametrize("name,data,opts", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_fp32c_gradient_and_loglik_with_multi_tile_chunks(name, data, opts, chunk_tiles):
    beta = random_beta(data.p, 0.3, seed=7)
    with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) as h:
        g1, g2 = h.gradient(beta)
        ll = h.loglik(beta)
    o1, o2 = oracle.grad_hess(data, beta)
    ol = oracle.loglik(data, beta)
    assert np.max(np.abs(g1 - o1)) <= 1e-5 * max(1.0, np.max(np.abs(o1)))
    assert np.max(np.abs(g2 - o2)) <= 1e-5 * max(1.0, np.max(np.abs(o2)))
    assert abs(ll - ol) <= 1e-7 * _ll_scale(data, beta, ol)


@pytest.mark.parametrize("chunk_tiles", (2, 5), indirect=True)
def test_fp32c_batch_with_multi_tile_chunks(chunk_tiles):
    """Uneven fits in one batched launch: each result within the FP32C tolerance of the oracle."""
    sets = [CASES[0], CASES[1], CASES[2]]
    hs = [cox.Handle(d, o, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) for _, d, o in sets]
    try:
        betas, infos = cox.batch_fit(hs)
    finally:
        for h in hs:
            h.close()
    for (name, d, o), b, i in zip(sets, betas, infos):
        ob, _ = _oracle_fit(name, d, o, i["sweeps"])
        ob2, oi2 = _oracle_fit(name, d, o)
        assert min(_rel_beta(b, ob), _rel_beta(b, ob2)) <= 1e-5, name
        assert abs(i["loglik"] - oi2["loglik"]) <= 1e-7 * _ll_scale(d, ob2, oi2["loglik"]), name


def test_chunk_tiles_knob_rejects_bad_values():
    with pytest.raises(cox.CoxError):
        cox.cox_debug_set_chunk_tiles(65)
    with pytest.raises(cox.CoxError):
        cox.cox_debug_set_chunk_tiles(-1)
    cox.cox_debug_set_chunk_tiles(0)


def _edge_cases():
    """The FP64 parity suite's edge cases (tests/test_gpu_parity.py), for the FP32C kernel."""
    from tests.test_gpu_parity import _edge_cases as edges
    return edges()


EDGES = _edge_cases()


@pytest.mark.parametrize("chunk_tiles", (0, 2), indirect=True)
@pytest.mark.parametrize("name,data,opts", EDGES, ids=[c[0] for c in EDGES])
def test_fp32c_edge_cases(name, data, opts, chunk_tiles):
    """No events, every row tied, singleton strata, a dense / empty / one-row column, tie heads on
    tile boundaries, head-capped tiles: the FP32C fit, gradient and log-likelihood against the
    oracle at the FP32C tolerances, with the library's chunk plan and with 2 tiles per chunk."""
    beta0 = random_beta(data.p, 0.2, seed=3)
    with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) as h:
        g1, g2 = h.gradient(beta0)
        ll = h.loglik(beta0)
        beta, info = h.fit()
    o1, o2 = oracle.grad_hess(data, beta0)
    ol = oracle.loglik(data, beta0)
    assert np.max(np.abs(g1 - o1)) <= 1e-5 * max(1.0, np.max(np.abs(o1))), name
    assert np.max(np.abs(g2 - o2)) <= 1e-5 * max(1.0, np.max(np.abs(o2))), name
    assert abs(ll - ol) <= 1e-7 * max(_ll_scale(data, beta0, ol), 1.0), name
    ob, _ = _oracle_fit(name, data, opts, info["sweeps"])
    ob2, oi2 = _oracle_fit(name, data, opts)
    if np.any(ob2):
        assert min(_rel_beta(beta, ob), _rel_beta(beta, ob2)) <= 1e-5, name
    else:
        assert np.max(np.abs(beta)) <= 1e-7, name
    assert abs(info["loglik"] - oi2["loglik"]) <= 1e-7 * max(_ll_scale(data, ob2, oi2["loglik"]), 1.0), name


# ---- the cached-S0 path: a step of a fit whose eta did not change since its previous step (that
#      step's update was 0) reads its tie groups' S0 from that step and computes column j's S1 (S2)
#      from the column's entries; with several chunks per CTA, CTAs take further chunks in list order
@pytest.fixture
def chunk_plan(request):
    cox.cox_set_chunk_plan(request.param)
    yield request.param
    cox.cox_set_chunk_plan(0)


def _l1_well_posed(name, data):
    """L1 at a quantile of |g'(0)| over the columns such that some coefficients stay at 0, at least
    two move, and none of those lands near 0 (at least 5 % of the largest): most steps leave eta
    unchanged, and no coefficient sits at the edge of the active set, where FP32 rounding of the
    gradient moves it by more than the FP32C tolerance."""
    g1, _ = oracle.grad_hess(data, np.zeros(data.p))
    for q in (0.5, 0.6, 0.7, 0.8, 0.9):
        opts = synth.CoxOptions(penalty=synth.PEN_L1, lam=float(np.quantile(np.abs(g1), q)), tol=1e-8)
        b, info = oracle.fit(data, opts)
        nz = np.abs(b[b != 0.0])
        if nz.size >= 2 and nz.size < data.p and nz.min() >= 0.05 * nz.max():
            _ORACLE[(name, None)] = (b, info)
            return name, data, opts
    raise AssertionError(f"{name}: no well-posed L1 weight")


_L1 = {}


def _l1_case(name):
    """The L1 cases, built on first use: one stratum, many strata, counting process, valued X."""
    if name not in _L1:
        base = {"many_strata_l1": CASES[1][1], "counting_l1": CASES[2][1], "dense_valued_l1": CASES[4][1]}
        _L1[name] = CASES[0] if name == "one_stratum_l1" else _l1_well_posed(name, base[name])
    return _L1[name]


L1_NAMES = ("one_stratum_l1", "many_strata_l1", "counting_l1", "dense_valued_l1")


@pytest.mark.parametrize("chunk_plan", (1, 3), indirect=True)
@pytest.mark.parametrize("chunk_tiles", (1, 2), indirect=True)
@pytest.mark.parametrize("case", L1_NAMES)
def test_fp32c_cached_s0_path_matches_oracle(case, chunk_tiles, chunk_plan):
    """L1 fits whose steps mostly leave eta unchanged, with one or three chunks per CTA, against the
    oracle at the FP32C tolerances."""
    name, data, opts = _l1_case(case)
    with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) as h:
        beta, info = h.fit()
    ob, _ = _oracle_fit(name, data, opts, info["sweeps"])
    ob2, oi2 = _oracle_fit(name, data, opts)
    assert np.any(ob2 == 0.0) and np.any(ob2 != 0.0), name   # the penalty keeps some coefficients at 0
    assert min(_rel_beta(beta, ob), _rel_beta(beta, ob2)) <= 1e-5, (name, chunk_tiles, chunk_plan)
    assert abs(info["loglik"] - oi2["loglik"]) <= 1e-7 * _ll_scale(data, ob2, oi2["loglik"]), name


@pytest.mark.parametrize("chunk_tiles", (2,), indirect=True)
def test_cached_s0_path_is_taken(chunk_tiles):
    """The same L1 fit with the cached-S0 path and without it: both within the FP32C tolerance of the
    oracle, and not bitwise equal (its S1 sums run in another order), so the path ran."""
    name, data, opts = _l1_case("many_strata_l1")
    out = []
    try:
        for enable in (True, False):
            cox.cox_debug_set_cached_s0(enable)
            with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) as h:
                out.append(h.fit())
    finally:
        cox.cox_debug_set_cached_s0(True)
    ob2, oi2 = _oracle_fit(name, data, opts)
    for beta, info in out:
        ob, _ = _oracle_fit(name, data, opts, info["sweeps"])
        assert min(_rel_beta(beta, ob), _rel_beta(beta, ob2)) <= 1e-5
    assert not np.array_equal(out[0][0], out[1][0])


@pytest.mark.parametrize("chunk_plan", (3,), indirect=True)
@pytest.mark.parametrize("chunk_tiles", (1, 2), indirect=True)
def test_fp32c_batch_cached_s0_and_chunk_plan(chunk_tiles, chunk_plan):
    """A batch of uneven L1 and L2 fits with three chunks per CTA: fits on the cached-S0 path and on
    the full pass share launches; each result within the FP32C tolerance of the oracle."""
    sets = [_l1_case("one_stratum_l1"), _l1_case("many_strata_l1"), _l1_case("counting_l1"), CASES[1],
            _l1_case("dense_valued_l1")]
    hs = [cox.Handle(d, o, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) for _, d, o in sets]
    try:
        betas, infos = cox.batch_fit(hs)
    finally:
        for h in hs:
            h.close()
    for (name, d, o), b, i in zip(sets, betas, infos):
        ob, _ = _oracle_fit(name, d, o, i["sweeps"])
        ob2, oi2 = _oracle_fit(name, d, o)
        assert min(_rel_beta(b, ob), _rel_beta(b, ob2)) <= 1e-5, name
        assert abs(i["loglik"] - oi2["loglik"]) <= 1e-7 * _ll_scale(d, ob2, oi2["loglik"]), name


def test_chunk_plan_knob_rejects_bad_values():
    with pytest.raises(cox.CoxError):
        cox.cox_set_chunk_plan(9)
    with pytest.raises(cox.CoxError):
        cox.cox_set_chunk_plan(-1)
    cox.cox_set_chunk_plan(0)


@pytest.mark.parametrize("chunk_tiles", (1, 2), indirect=True)
@pytest.mark.parametrize("case", ("many_strata_l1", "counting_l1", "dense_valued_l1"))
def test_gradient_on_the_cached_s0_path(case, chunk_tiles):
    """cox_gradient evaluates every column at one eta: its launches after the first read the tie
    groups' S0 kept from the first. With and without that path the gradient and the Hessian
    diagonal match the oracle at the FP32C tolerance; on binary X the two differ in their last bits
    (the path's S1 sums run in another order), so the path ran."""
    _, data, opts = _l1_case(case)
    beta = random_beta(data.p, 0.3, seed=11)
    out = []
    try:
        for enable in (True, False):
            cox.cox_debug_set_cached_s0(enable)
            with cox.Handle(data, opts, precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM) as h:
                out.append(h.gradient(beta))
    finally:
        cox.cox_debug_set_cached_s0(True)
    o1, o2 = oracle.grad_hess(data, beta)
    for g1, g2 in out:
        assert np.max(np.abs(g1 - o1)) <= 1e-5 * max(1.0, np.max(np.abs(o1))), case
        assert np.max(np.abs(g2 - o2)) <= 1e-5 * max(1.0, np.max(np.abs(o2))), case
    if data.val is None:
        assert not np.array_equal(out[0][0], out[1][0]), case
