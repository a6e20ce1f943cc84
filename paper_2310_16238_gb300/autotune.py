"""Tile-length autotuner for batched fits (streaming coordinate-step kernel).

For a set of data sets and a precision, it times a short batched run (a bounded number of
coordinate steps) at each candidate tile length and returns the fastest. Results are cached
per (precision, total-rows bucket) for the life of the process. All timing runs go through the
C ABI (cox_batch_fit); nothing here computes on the CPU.
"""
from __future__ import annotations

import math
import time

from . import cox, synth

_CACHE = {}
CANDIDATES = {cox.COX_FP64: (2048, 4096), cox.COX_FP32C: (2048, 4096)}


def batch_tile(sets, precision, max_sweeps_probe: int = 1) -> int:
    """Best tile length for fitting every (data, options) pair of ``sets`` together."""
    rows = sum(d.n for d, _ in sets)
    key = (precision, int(math.log2(max(rows, 1))))
    if key in _CACHE:
        return _CACHE[key]
    best, best_t = None, float("inf")
    for tile in CANDIDATES[precision]:
        handles = []
        for d, olist in sets:
            o = olist[0]
            probe = synth.CoxOptions(penalty=o.penalty, lam=o.lam, l2_var=o.l2_var, tol=0.0,
                                     max_sweeps=max_sweeps_probe)
            handles.append(cox.Handle(d, probe, precision=precision, tile=tile, engine=cox.COX_ENGINE_STREAM))
        cox.batch_fit(handles)           # warm-up (graph capture, caches)
        t0 = time.perf_counter()
        cox.batch_fit(handles)
        dt = time.perf_counter() - t0
        for h in handles:
            h.close()
        if dt < best_t:
            best, best_t = tile, dt
    _CACHE[key] = best
    return best
