"""Seeded synthetic inputs generated on the GPU with torch, for workloads too large to draw in
NumPy within a benchmark's time (serving requests of up to 1e7 rows and 2e9 nonzeros).

The recipes are those of ``synth.stratified_sparse`` and ``synth.time_varying`` (the same
distributions, strata, event models and sort order), drawn with torch's generator instead of
NumPy's, so the data differ from the NumPy draws of the same seed. Two simplifications, both
within the recipes' own tolerances: a column's rows are drawn with replacement and merged (for
densities up to 1e-2 this loses at most ~0.5 % of its entries), and the event-rate bisection runs
for 50 steps. This module holds no Cox arithmetic: it only draws inputs, which the library then
copies from device memory. Nothing here is used by the oracle or its tests.
"""
from __future__ import annotations

import math

import numpy as np

from . import synth


def _bisect(f, lo, hi, target, iters=50):
    a, b = math.log(lo), math.log(hi)
    for _ in range(iters):
        m = 0.5 * (a + b)
        if f(math.exp(m)) < target:
            a = m
        else:
            b = m
    return math.exp(0.5 * (a + b))


def _columns(torch, gen, n_rows, p, dens, dev):
    """Binary columns: column j holds ~Binomial(n_rows, dens[j]) distinct rows. Returns the
    column of each entry and its (unsorted) row, both int64, duplicates removed."""
    counts = torch.binomial(torch.full((p,), float(n_rows), dtype=torch.float64, device=dev),
                            torch.as_tensor(dens, dtype=torch.float64, device=dev), generator=gen).to(torch.int64)
    total = int(counts.sum().item())
    col = torch.repeat_interleave(torch.arange(p, device=dev, dtype=torch.int64), counts)
    row = torch.randint(0, n_rows, (total,), generator=gen, device=dev, dtype=torch.int64)
    key = torch.unique(col * n_rows + row)          # sorted, duplicates merged
    return key // n_rows, key % n_rows


def _finalize(torch, stop, event, stratum, start, col, row, p, dev):
    """Sort rows by (stratum, stop, original index) and build the CSC over the sorted rows."""
    n = stop.shape[0]
    key = stop.to(torch.int64)
    if stratum is not None:
        key = stratum.to(torch.int64) * (1 << 20) + key
    order = torch.sort(key, stable=True).indices
    newpos = torch.empty_like(order)
    newpos[order] = torch.arange(n, device=dev, dtype=torch.int64)
    k2 = torch.sort(col * n + newpos[row]).values
    col_s = k2 // n
    row_idx = (k2 - col_s * n).to(torch.int32)
    counts = torch.bincount(col_s, minlength=p)
    col_ptr = torch.zeros(p + 1, dtype=torch.int64, device=dev)
    col_ptr[1:] = torch.cumsum(counts, 0)
    return synth.CoxData(stop=stop[order].to(torch.int32).contiguous(), event=event[order].to(torch.uint8).contiguous(),
                         stratum=None if stratum is None else stratum[order].to(torch.int32).contiguous(),
                         start=None if start is None else start[order].to(torch.int32).contiguous(),
                         col_ptr=col_ptr, row_idx=row_idx.contiguous(), p=p, recipe="device")


def stratified_sparse(n, p, k, density, seed, dev, n_support=20, event_frac=0.05, admin_days=3650, shape=1.5):
    """``synth.stratified_sparse`` on the device with one density for every column."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    k = max(1, min(k, n))
    sizes = torch.as_tensor(synth._sizes_zipf(n, k), device=dev)
    stratum = torch.repeat_interleave(torch.arange(k, device=dev, dtype=torch.int64), sizes)
    col, row = _columns(torch, gen, n, p, np.full(p, density), dev)
    sup = torch.randperm(p, generator=gen, device=dev)[:min(n_support, p)]
    beta = torch.zeros(p, dtype=torch.float64, device=dev)
    beta[sup] = 0.3 * torch.randn(len(sup), generator=gen, device=dev, dtype=torch.float64)
    eta = torch.zeros(n, dtype=torch.float64, device=dev)
    eta.index_add_(0, row, beta[col])
    u = torch.rand(n, generator=gen, device=dev, dtype=torch.float64).clamp_min(1e-300)
    base = -torch.log(u) / torch.exp(eta)
    h = _bisect(lambda hh: float(((base / hh) ** (1.0 / shape) <= admin_days).double().mean().item()), 1e-12, 1e3,
                event_frac)
    t = (base / h) ** (1.0 / shape)
    ev = (t <= admin_days)
    y = torch.clamp(torch.ceil(torch.clamp(t, max=float(admin_days))), min=1).to(torch.int64)
    return _finalize(torch, y, ev, stratum, None, col, row, p, dev)


def time_varying(n_subj, p, k, density, seed, dev, n_support=20, event_frac=0.10, max_intervals=20):
    """``synth.time_varying`` on the device: counting-process rows with per-interval covariates."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    i64, f64 = torch.int64, torch.float64
    fu = torch.randint(30, 3651, (n_subj,), generator=gen, device=dev, dtype=i64)
    lam = torch.full((n_subj,), 2.0, device=dev, dtype=f64)
    m = torch.clamp(torch.poisson(lam, generator=gen).to(i64) + 1, max=max_intervals)
    ncut = m - 1
    subj_of_cut = torch.repeat_interleave(torch.arange(n_subj, device=dev, dtype=i64), ncut)
    cut_day = 1 + torch.floor(torch.rand(subj_of_cut.shape[0], generator=gen, device=dev, dtype=f64)
                              * (fu[subj_of_cut] - 1)).to(i64)
    key = torch.unique(subj_of_cut * 4096 + cut_day)   # sorted by (subject, day); duplicate days merged
    subj_of_cut, cut_day = key // 4096, key % 4096
    ncut = torch.bincount(subj_of_cut, minlength=n_subj)
    nrow = ncut + 1
    r_total = int(nrow.sum().item())
    subj = torch.repeat_interleave(torch.arange(n_subj, device=dev, dtype=i64), nrow)
    first = torch.zeros(n_subj + 1, dtype=i64, device=dev)
    first[1:] = torch.cumsum(nrow, 0)
    is_last = torch.zeros(r_total, dtype=torch.bool, device=dev)
    is_last[first[1:] - 1] = True
    is_first = torch.zeros(r_total, dtype=torch.bool, device=dev)
    is_first[first[:-1]] = True
    stop = torch.empty(r_total, dtype=i64, device=dev)
    start = torch.empty(r_total, dtype=i64, device=dev)
    stop[~is_last] = cut_day
    stop[is_last] = fu
    start[is_first] = 0
    start[~is_first] = cut_day
    col, row = _columns(torch, gen, r_total, p, np.full(p, density), dev)
    sup = torch.randperm(p, generator=gen, device=dev)[:min(n_support, p)]
    beta = torch.zeros(p, dtype=f64, device=dev)
    beta[sup] = 0.3 * torch.randn(len(sup), generator=gen, device=dev, dtype=f64)
    eta = torch.zeros(r_total, dtype=f64, device=dev)
    eta.index_add_(0, row, beta[col])
    w = torch.exp(eta) * (stop - start).to(f64)     # cumulative hazard per row, per unit h
    cumw = torch.cumsum(w, 0)
    subj_w = torch.zeros(n_subj, dtype=f64, device=dev).index_add_(0, subj, w)
    e_draw = -torch.log(torch.rand(n_subj, generator=gen, device=dev, dtype=f64).clamp_min(1e-300))
    h = _bisect(lambda hh: float((e_draw < hh * subj_w).double().mean().item()), 1e-12, 1e3, event_frac)
    before = cumw - w
    target = before[first[:-1]] + e_draw / h
    has_ev = e_draw < h * subj_w
    ev_row = torch.searchsorted(cumw, target, side="left")
    ev_row = torch.where(has_ev, torch.minimum(ev_row, first[1:] - 1), torch.full_like(ev_row, -1))
    event = torch.zeros(r_total, dtype=torch.uint8, device=dev)
    sel = torch.nonzero(has_ev).squeeze(1)
    er = ev_row[sel]
    t_ev = start[er].to(f64) + (target[sel] - before[er]) / (h * torch.exp(eta[er]))
    new_stop = torch.minimum(torch.maximum(torch.ceil(t_ev).to(i64), start[er] + 1), stop[er])
    stop[er] = new_stop
    event[er] = 1
    last_keep = torch.where(has_ev, ev_row, first[1:] - 1)
    pos_in = torch.arange(r_total, device=dev, dtype=i64) - first[subj]
    keep_row = pos_in <= (last_keep[subj] - first[subj])
    old_to_new = torch.full((r_total,), -1, dtype=i64, device=dev)
    nk = int(keep_row.sum().item())
    old_to_new[keep_row] = torch.arange(nk, device=dev, dtype=i64)
    kept = keep_row[row]
    col, row = col[kept], old_to_new[row[kept]]
    stratum_subj = torch.randint(0, k, (n_subj,), generator=gen, device=dev, dtype=i64)
    return _finalize(torch, stop[keep_row], event[keep_row], stratum_subj[subj[keep_row]], start[keep_row],
                     col, row, p, dev)


def request_data(req: "synth.Request", dev):
    """Device data and options of one serving request (the recipe of ``synth.request_data``
    without a row cap: counting-process requests use n_subj / 3 subjects)."""
    if req.counting:
        data = time_varying(max(10, req.n_subj // 3), req.p, req.k, req.density, req.seed, dev,
                            n_support=min(20, req.p))
    else:
        data = stratified_sparse(req.n_subj, req.p, req.k, req.density, req.seed, dev, n_support=min(20, req.p))
    if req.penalty == synth.PEN_L1:
        opts = synth.CoxOptions(penalty=synth.PEN_L1, lam=1e-4 * data.n, tol=1e-8)
    else:
        opts = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=1.0, tol=1e-8)
    return data, opts
