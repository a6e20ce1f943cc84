"""Schedule autotuner for batched fits (streaming coordinate-step kernels).

For a set of data sets and a precision it times short batched runs (at most two sweeps) at each
candidate schedule and returns the fastest:
  * FP64 streaming kernel: the tile length (positions per work item);
  * FP32C chunked kernel: the chunks per resident CTA of its plans (one chunk per CTA, or several
    taken in work-list order, so that CTAs freed by cheap chunks take others). Its tiles are fixed
    at 4,096 positions.
Results are cached per (precision, total-rows bucket, fits) for the life of the process. All
timing runs go through the C ABI (cox_batch_fit); nothing here computes on the CPU.
"""
from __future__ import annotations

import math
import time

from . import cox, synth

_CACHE = {}
CANDIDATES = {cox.COX_FP64: (2048, 4096), cox.COX_FP32C: (4096,)}
PLAN_CANDIDATES = (1, 2, 3)


def _probe_handles(sets, precision, tile, every_option):
    """Every fit (every option of each set when every_option, else its first) for at most two
    sweeps with its own tolerance: the first sweep of every fit and the second of those that go on,
    as in the batch itself."""
    handles = []
    for d, olist in sets:
        probe = [synth.CoxOptions(penalty=o.penalty, lam=o.lam, l2_var=o.l2_var, tol=o.tol, max_sweeps=2)
                 for o in (olist if every_option else olist[:1])]
        base = cox.Handle(d, probe[0], precision=precision, tile=tile, engine=cox.COX_ENGINE_STREAM)
        handles.append(base)
        handles.extend(base.clone(o) for o in probe[1:])
    return handles


def _time_batch(handles):
    cox.batch_fit(handles)           # warm-up (graph capture, caches)
    t0 = time.perf_counter()
    cox.batch_fit(handles)
    return time.perf_counter() - t0


def batch_tile(sets, precision) -> int:
    """Best tile length for fitting every (data, options) pair of ``sets`` together."""
    if len(CANDIDATES[precision]) == 1:
        return CANDIDATES[precision][0]
    rows = sum(d.n for d, _ in sets)
    key = (precision, int(math.log2(max(rows, 1))))
    if key in _CACHE:
        return _CACHE[key]
    best, best_t = None, float("inf")
    for tile in CANDIDATES[precision]:
        handles = _probe_handles(sets, precision, tile, every_option=False)
        dt = _time_batch(handles)
        for h in handles:
            h.close()
        if dt < best_t:
            best, best_t = tile, dt
    _CACHE[key] = best
    return best


def batch_chunk_plan(sets) -> int:
    """Best number of chunks per resident CTA for fitting every (data, options) pair of ``sets``
    together with the FP32C kernel, set process-wide (cox_set_chunk_plan) and returned. Every fit
    runs in the probe (the mix of steps that read cached S0 and full passes is the batch's own)."""
    rows = sum(d.n * len(ol) for d, ol in sets)
    key = ("plan", int(math.log2(max(rows, 1))), sum(len(ol) for _, ol in sets))
    if key not in _CACHE:
        best, best_t = None, float("inf")
        for k in PLAN_CANDIDATES:
            cox.cox_set_chunk_plan(k)
            handles = _probe_handles(sets, cox.COX_FP32C, 4096, every_option=True)
            dt = _time_batch(handles)
            for h in handles:
                h.close()
            if dt < best_t:
                best, best_t = k, dt
        _CACHE[key] = best
    cox.cox_set_chunk_plan(_CACHE[key])
    return _CACHE[key]
