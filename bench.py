"""Benchmark: regularized stratified Cox CCD fits on GB300 (one JSON line on rank 0).

Default workload (the headline): the large stratified sparse fit -- N = 2,000,000 subjects,
p = 2,000 binary columns with log-uniform density in [1e-4, 5e-2], 100 Zipf(1.1) strata,
Weibull(1.5) event times in integer days (~5 % events), L1 gamma = 1e-3 N, FP64 precision,
seeded synthetic data. A step is one complete fit through the C ABI: cox_create
(device-resident inputs: validation, strata, tie groups, delta'X, tile plan) + cox_fit (CCD
sweeps until the tolerance) + cox_destroy. The metric is coordinate updates per second.

At that L1 weight every coefficient stays at 0 (the fit ends after one sweep and no eta update
runs), so the same line also carries, as sub-results measured in the same run:
  moving   the same data at gamma = 1e-5 N (hundreds of coefficients move), timed to
           convergence, with the error of its two-sweep iterate against the FP64 oracle;
  batch    256 fits (4 outcomes x 4 folds x 16 L1 weights over one shared X): the plain
           one-fit-at-a-time FP64 path against the batched launches (compensated FP32
           streaming, FP64 streaming, FP64 incremental waves), with the HBM roofline of the
           batched streaming kernel;
  counting_process  the counting-process fit (1e6 subjects, ~2.9e6 (start, stop] rows, p = 5000,
           K = 20, L2), timed per fit;
  plain    the small dense fit (N = 1000, p = 10), whole fits per step, against the FP64 oracle's;
  serving  Poisson fit requests (rows logU[1e4, 1e7], p logU[100, 2e4], density logU[1e-4,
           1e-2], 1-200 strata, half counting-process, L1 / L2) into the continuous-batching
           server: its capacity under a burst, then a stream at a sustainable rate with
           p50 / p99 time-to-fit.

Timing: W warm-up steps, then K steps, each bracketed by CUDA events on the fit's stream; L2
(129 MB) is flushed by writing a 512 MB buffer before every timed step (outside the events);
barrier + synchronize on both sides; max over ranks. Multi-GPU (torchrun): every rank fits its
own independent replica (weak scaling, no collective on the data path).

`--impl reference` times the FP64 CPU oracle (the plain restatement of the paper's method) on the
box's host cores: one independent oracle process per usable core, each running the same bounded
sample (a fixed number of coordinate updates of the same fit from beta = 0).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import multiprocessing as mp
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_16238_gb300 import synth  # noqa: E402

METRIC = "coordinate updates/sec and fits/sec vs plain FP64 path; HBM roofline %; p99 latency"
EXCHANGE_FLOOR_US = 0.87   # cross-SM flag round trip on GB300 (a step of one fit needs at least one)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def hbm_peak():
    p = _peaks()
    if "hbm_gbs" in p:
        return float(p["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    return 6800.0, "profiling recipe fallback 6.8 TB/s (of fallback)"


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


ENGINE_NAMES = {1: "streaming", 2: "resident", 3: "incremental"}

# DRAM bytes (read + write) per coordinate step of a kernel, from one ncu capture of the same kernel
# on the same workload (launch total / steps it ran; the captures run `bench.py --workload probe`).
# Keyed by (engine, workload, precision); absent = not captured for the current kernel.
TRAFFIC = {
    # --probe incr: 156.02 MB read + 33.95 MB written per 1-sweep launch of 2001 steps
    ("incremental", "stratified_sparse", "fp64"): (156.023e6 + 33.954e6) / 2001,
    # --probe stream_fp32c: an evaluation launch (a fit's launch adds the previous column's update, ~0.2 MB)
    ("streaming", "time_varying", "fp32c"): 25.52e6,
    # --probe stream_fp64: an evaluation launch
    ("streaming", "time_varying", "fp64"): 47.03e6,
}


def aggregate_ranks(units_per_rank: float, ms_per_step: float, world: int, device):
    """Whole-job throughput over replicas: every rank processed `units_per_rank` per step; the
    job's step time is the slowest rank's (max over ranks)."""
    slowest = float(ms_per_step)
    if world > 1:
        import torch
        t = torch.tensor([ms_per_step], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        slowest = float(t.item())
    return units_per_rank * world / (slowest * 1e-3), slowest


def headline_workload(scale: float = 1.0, seed_offset: int = 0):
    n = int(2_000_000 * scale)
    data, opts = synth.stratified_sparse(n=n, p=2000, k=100, seed=synth.SEED_BASE + 2 + seed_offset)
    name = f"stratified_sparse N={n} p=2000 K=100 binary density logU[1e-4,5e-2] L1 gamma=1e-3*N"
    return data, opts, name


def moving_options(n: int):
    return synth.CoxOptions(penalty=synth.PEN_L1, lam=1e-5 * n, tol=1e-8)


def headline_config(wname: str) -> dict:
    """The workload the metric is quoted on (identical in both arms)."""
    return {"workload": wname,
            "precision": "FP64-level results: tolerance vs the FP64 oracle 1e-9 beta, 1e-11 log-likelihood (the GPU "
                         "path sums in double-word FP32, about 48-bit significands, with FP64 eta, beta and step; "
                         "`dtype` gives each arm's arithmetic)"}


def dense_bytes_per_step(M: int, G: int, K: int, nnz_pos: float, s_e: int, moved: bool) -> float:
    """Algorithmic bytes of one coordinate step of the paper's dense method (the risk sequence of
    exp(eta) read once, the tie-group and stratum tables, column j's entries, and -- when the
    previous coordinate moved -- its entries' eta read and written and exp(eta) written)."""
    return s_e * M + 8.0 * G + 4.0 * (K + 1) + 4.0 * nnz_pos + ((4 + 16 + s_e) * nnz_pos if moved else 0.0)


def incr_own_bytes_per_step(M: int, p: int, nnz_pos: float, s_e: int, moved: bool) -> float:
    """Bytes the incremental kernel itself moves per coordinate step: column j's entries with eta and
    v (read and, when the step moved, written) plus the dense refresh once per sweep."""
    return (4.0 + 16.0) * nnz_pos + (16.0 * nnz_pos if moved else 0.0) + (8.0 + 8.0 + s_e) * M / p


def dtype_of(engine, s_e):
    """Arithmetic of the path: the incremental engine sums in double-word FP32 (about 48 bits) with
    FP64 eta, beta and step; the dense engines in FP64, or FP32 with compensation and FP64 carries."""
    if engine == "incremental":
        return "f32x2+f64"
    return "f64" if s_e == 8 else "f32+f64"


def roofline_of(engine, data, beta, G, K, s_e, step_us, wname, precision_name):
    """Roofline of the coordinate-step kernel against the measured HBM copy bandwidth: `achieved` =
    the kernel's algorithmic bytes per coordinate step x the steps one launch runs / the launch's
    CUDA-event time. A dense engine's bytes are the paper's dense scan (every position read); the
    incremental kernel's are its own (column j's entries and the changed positions), with the
    latency floor of its step beside them and, labelled effective, the bandwidth the dense scan
    would need to match its step time."""
    M = data.n if data.start is None else 2 * data.n
    nnz_mean = float(np.diff(data.col_ptr).mean())
    nnz_pos = nnz_mean * (2.0 if data.start is not None else 1.0)
    moved = bool(np.count_nonzero(beta) > 0)
    peak, src = hbm_peak()
    dense = dense_bytes_per_step(M, G, K, nnz_pos, s_e, moved)
    dense_gbs = dense / (step_us * 1e-6) / 1e9
    traffic = TRAFFIC.get((engine, wname.split()[0], precision_name))
    if engine != "incremental":
        return {"bound": "hbm", "achieved": dense_gbs, "peak": peak, "unit": "GB/s", "frac": dense_gbs / peak,
                "traffic": traffic, "kernel": f"coordinate step ({engine})", "step_us": step_us,
                "alg_bytes_per_step": dense,
                "basis": "bytes of the paper's dense scan per coordinate step x steps per launch / launch time",
                "peak_source": src}
    own = incr_own_bytes_per_step(M, data.p, nnz_pos, s_e, moved)
    own_gbs = own / (step_us * 1e-6) / 1e9
    return {"bound": "hbm", "achieved": own_gbs, "peak": peak, "unit": "GB/s", "frac": own_gbs / peak,
            "traffic": traffic, "kernel": "coordinate step (incremental)", "step_us": step_us,
            "alg_bytes_per_step": own,
            "basis": "the incremental kernel's own bytes per coordinate step (column j's entries with eta "
                     "and v, the update's writes, the dense refresh once per sweep) / step time",
            "peak_source": src,
            "binding": "latency, not bytes: a step is a chain of barrier-separated phases around one "
                       "cross-SM exchange",
            "latency": {"step_us": step_us, "floor_us": EXCHANGE_FLOOR_US, "frac": EXCHANGE_FLOOR_US / step_us,
                        "floor": "one cross-SM exchange round trip per coordinate step"},
            "effective_dense": {"achieved": dense_gbs, "frac": dense_gbs / peak, "alg_bytes_per_step": dense,
                                "note": "effective, not moved: the bandwidth the paper's dense scan (every "
                                        "position read per step) would need to match this step time"}}


def _device_copy(data, dev):
    import torch
    ddev = synth.CoxData(**{**data.__dict__})
    for f in ("stop", "start", "event", "stratum", "col_ptr", "row_idx", "val"):
        a = getattr(data, f)
        if a is not None:
            setattr(ddev, f, torch.from_numpy(np.ascontiguousarray(a)).to(dev))
    return ddev


def _timed_fits(cox, ddev, opts, precision, stream, flush, steps, warmup, clk=None):
    """CUDA-event times of `steps` whole fits (create + fit + destroy), L2 flushed before each."""
    import torch

    def step():
        h = cox.cox_create(ddev, opts, precision=precision, stream=stream.cuda_stream)
        try:
            return cox.cox_fit(h)
        finally:
            cox.cox_destroy(h)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    torch.cuda.synchronize()
    times, infos, beta = [], [], None
    launches0 = cox.cox_launch_count()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            beta, info = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
    torch.cuda.synchronize()
    return times, infos, beta, cox.cox_launch_count() - launches0


def run_headline(args, rank, world, local_rank):
    import torch
    from paper_2310_16238_gb300 import cox
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    data, opts, wname = headline_workload(args.scale, rank)
    precision = cox.COX_FP64
    stream = torch.cuda.Stream(device=dev)
    ddev = _device_copy(data, dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    h = cox.cox_create(ddev, opts, precision=precision, stream=stream.cuda_stream)
    md = cox.cox_metadata(h)
    G, K = len(md["group_time"]), len(md["strata_start"]) - 1
    cox.cox_destroy(h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local_rank) as clk:
        times, infos, beta, launches = _timed_fits(cox, ddev, opts, precision, stream, flush, args.steps, args.warmup)
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    step_ms = float(np.mean(times))
    coords = float(np.mean([i["coord_updates"] for i in infos]))
    steps_run = float(np.sum([i["coord_updates"] + 1 for i in infos]))
    step_us = float(np.sum([i["sweep_ms"] for i in infos])) / steps_run * 1e3
    engine = ENGINE_NAMES.get(infos[-1]["engine"], "unknown")
    value, slowest_ms = aggregate_ranks(coords, step_ms, world, dev)
    result = {
        "metric": METRIC, "value": value, "unit": "coord_updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": slowest_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_of(engine, 8), "data": "synthetic (seeded; paper cohorts unavailable)",
        "config": headline_config(wname),
        "parallelism": f"replicas{world}",
        "fit": {"engine": engine, "sweeps": infos[-1]["sweeps"], "coord_updates_per_fit": coords,
                "nonzero_beta": int(np.count_nonzero(beta)), "tie_groups": G, "strata": K,
                "fits_per_s": world / (slowest_ms * 1e-3), "step_us": step_us,
                "l2": "flushed before every step (512 MB write)",
                "note": "at this L1 weight every coefficient stays at 0 (one sweep, no eta update); "
                        "`moving` is the same data at a weight where coefficients move"},
        "roofline": roofline_of(engine, data, beta, G, K, 8, step_us, wname, "fp64"),
        "gpu_launches": int(launches), "wall_s": wall, "clocks": clk.summary(),
    }
    return result, (data, ddev, stream, flush, G, K)


def run_moving(args, data, ddev, stream, flush, G, K, oracle_result):
    """The headline data at gamma = 1e-5 N: timed fits to convergence, plus the error of the
    two-sweep iterate against the FP64 oracle's."""
    from paper_2310_16238_gb300 import cox
    opts = moving_options(data.n)
    with ClockSampler(0) as clk:
        times, infos, beta, _ = _timed_fits(cox, ddev, opts, cox.COX_FP64, stream, flush, max(3, args.steps // 4), 1)
    ms = float(np.mean(times))
    coords = float(np.mean([i["coord_updates"] for i in infos]))
    steps_run = float(np.sum([i["coord_updates"] + 1 for i in infos]))
    step_us = float(np.sum([i["sweep_ms"] for i in infos])) / steps_run * 1e3
    engine = ENGINE_NAMES.get(infos[-1]["engine"], "unknown")
    out = {"workload": f"stratified_sparse N={data.n} p={data.p} K=100 L1 gamma=1e-5*N (same data as the headline)",
           "engine": engine, "dtype": dtype_of(engine, 8), "fits": len(times), "ms_per_fit": ms,
           "fits_per_s": 1e3 / ms, "coord_updates_per_s": coords / (ms * 1e-3), "sweeps": infos[-1]["sweeps"],
           "converged": bool(infos[-1]["converged"]), "nonzero_beta": int(np.count_nonzero(beta)),
           "step_us": step_us,
           "roofline": roofline_of(engine, data, beta, G, K, 8, step_us, "stratified_sparse_moving", "fp64"),
           "clocks": clk.summary()}
    # the two-sweep iterate of the same fit, compared with the oracle's (computed beside the GPU legs)
    o2 = synth.CoxOptions(penalty=opts.penalty, lam=opts.lam, tol=0.0, max_sweeps=2)
    h = cox.cox_create(ddev, o2, precision=cox.COX_FP64, stream=stream.cuda_stream)
    try:
        b2, i2 = cox.cox_fit(h)
        dx = cox.cox_dx(h)
    finally:
        cox.cox_destroy(h)
    if oracle_result is not None:
        ob, oll = oracle_result
        scale = max(abs(oll), float(np.sum(np.abs(ob) * np.abs(dx))) + float(np.sum(data.event)))
        out["vs_oracle"] = {"sweeps": 2, "max_rel_beta_err": float(np.max(np.abs(b2 - ob)) / max(np.max(np.abs(ob)), 1e-300)),
                            "rel_loglik_err": abs(i2["loglik"] - oll) / scale, "tolerance": {"beta": 1e-9, "loglik": 1e-11},
                            "oracle": "FP64 CPU oracle, the same fit after 2 sweeps (element by element)"}
    return out


def run_plain(args, stream, oracle_result):
    """The small dense workload (N = 1000, p = 10 dense N(0,1) covariates, one stratum, L2): whole
    fits (cox_create from host arrays + cox_fit + cox_destroy) per step, and the fit against the
    FP64 oracle's at the same sweep count."""
    import torch
    from paper_2310_16238_gb300 import cox
    data, opts = synth.plain_dense()
    times, info, beta = [], None, None
    for k in range(13):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = cox.cox_create(data, opts, precision=cox.COX_FP64, stream=stream.cuda_stream)
        beta, info = cox.cox_fit(h)
        cox.cox_destroy(h)
        e1.record(stream)
        e1.synchronize()
        if k >= 3:
            times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    engine = ENGINE_NAMES.get(info["engine"], "unknown")
    out = {"workload": "plain_dense N=1000 p=10 dense N(0,1), 1 stratum, L2 var=1, tol 1e-8", "engine": engine,
           "dtype": dtype_of(engine, 8), "fits": len(times), "ms_per_fit": ms, "fits_per_s": 1e3 / ms,
           "coord_updates_per_s": info["coord_updates"] / (ms * 1e-3), "sweeps": info["sweeps"]}
    if oracle_result is not None:
        ob, oll, osw = oracle_result
        out["vs_oracle"] = {"sweeps_gpu": int(info["sweeps"]), "sweeps_oracle": osw,
                            "max_rel_beta_err": float(np.max(np.abs(beta - ob)) / max(np.max(np.abs(ob)), 1e-300)),
                            "rel_loglik_err": abs(info["loglik"] - oll) / max(abs(oll), float(np.sum(data.event))),
                            "tolerance": {"beta": 1e-9, "loglik": 1e-11},
                            "oracle": "FP64 CPU oracle, the same fit to convergence"}
    return out


# ---------------------------------------------------------------- config 4: batched fits
def run_batch(args, sub=False):
    """256 fits (4 outcomes x 4 folds x 16 L1 weights) over one shared binary X: the plain
    one-fit-at-a-time FP64 path against the batched launches."""
    import torch
    from paper_2310_16238_gb300 import autotune, cox
    sets = synth.batch_views(n_total=int(1_000_000 * args.scale), n_lo=1e4 * args.scale, n_hi=1e6 * args.scale)
    stream = torch.cuda.Stream()
    n_fits = sum(len(ol) for _, ol in sets)
    rows = int(sum(d.n * len(ol) for d, ol in sets))
    out = {"workload": f"batch_views: shared binary X {int(1e6 * args.scale)}x1000 density 1e-2, 16 training sets "
                       f"(4 outcomes x 4 folds) N~logU[1e4,1e6] with 1-50 strata, 16 L1 weights each",
           "fits": n_fits, "rows_total": rows}
    meta = []
    for d, ol in sets:
        h = cox.Handle(d, ol[0], precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM)
        md = h.metadata()
        meta.append((len(md["group_time"]), len(md["strata_start"]) - 1, float(np.diff(d.col_ptr).mean())))
        h.close()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, time.perf_counter() - t0, e0.elapsed_time(e1)

    # the plain path: every fit on its own, one after the other (AUTO engine, FP64)
    def plain():
        res = []
        for d, ol in sets:
            for o in ol:
                with cox.Handle(d, o, precision=cox.COX_FP64, stream=stream.cuda_stream) as h:
                    res.append(h.fit())
        return res
    with ClockSampler(0) as clk:
        ref, sec, _ = timed(plain)
    out["plain_fp64"] = {"fits_per_s": n_fits / sec, "seconds": sec, "engine": "AUTO per fit (one fit at a time)",
                         "clocks": clk.summary()}

    flat = [(d, o) for d, ol in sets for o in ol]

    def errors(betas, infos):
        """Largest beta error relative to the fit's max |beta| against the plain FP64 fit stopped
        at the same sweep (a fit whose convergence test passed one sweep earlier or later in the
        other precision is refitted in FP64 for that many sweeps, untimed)."""
        eb, mism = 0.0, 0
        for k, (bb, ii, (b, i)) in enumerate(zip(betas, infos, ref)):
            if ii["sweeps"] != i["sweeps"]:
                mism += 1
                d, o = flat[k]
                o2 = dataclasses.replace(o, max_sweeps=int(ii["sweeps"]), tol=0.0)
                with cox.Handle(d, o2, precision=cox.COX_FP64, stream=stream.cuda_stream) as h:
                    b, _ = h.fit()
            den = max(np.max(np.abs(b)), 1e-12) if np.any(b) else 1.0
            eb = max(eb, float(np.max(np.abs(bb - b)) / den))
        return eb, mism

    peak, src = hbm_peak()
    for prec, name, engine in ((cox.COX_FP32C, "batched_fp32c", cox.COX_ENGINE_STREAM),
                               (cox.COX_FP64, "batched_fp64", cox.COX_ENGINE_STREAM),
                               (cox.COX_FP64, "batched_incremental", cox.COX_ENGINE_AUTO)):
        tile = autotune.batch_tile(sets, prec) if engine == cox.COX_ENGINE_STREAM else 0
        plan = autotune.batch_chunk_plan(sets) if prec == cox.COX_FP32C and engine == cox.COX_ENGINE_STREAM else None
        handles = []
        for d, ol in sets:
            base = cox.Handle(d, ol[0], precision=prec, tile=tile, engine=engine, stream=stream.cuda_stream)
            handles.append(base)
            handles.extend(base.clone(o) for o in ol[1:])
        launches0 = cox.cox_launch_count()
        with ClockSampler(0) as clk:
            (betas, infos), sec, dev_ms = timed(lambda: cox.batch_fit(handles))
        launches = cox.cox_launch_count() - launches0
        err, mism = errors(betas, infos)
        r = {"fits_per_s": n_fits / sec, "seconds": sec, "device_ms": dev_ms,
             "engine": ENGINE_NAMES.get(infos[0]["engine"], "unknown"), "tile": tile or None,
             "chunks_per_cta": plan,
             "max_rel_beta_err_vs_plain_fp64": err, "sweep_mismatches_vs_plain_fp64": mism,
             "gpu_launches": int(launches),
             "speedup_vs_plain": (n_fits / sec) / out["plain_fp64"]["fits_per_s"], "clocks": clk.summary()}
        if engine == cox.COX_ENGINE_STREAM:
            s_e = 4 if prec == cox.COX_FP32C else 8
            alg = 0.0
            for k, ((d, ol), (G, K, nnz)) in enumerate(zip(sets, meta)):
                for m in range(len(ol)):
                    i = infos[k * len(ol) + m]
                    steps = i["coord_updates"] + 1
                    alg += steps * dense_bytes_per_step(d.n, G, K, nnz, s_e, True)
            ach = alg / (dev_ms * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                             "alg_bytes": alg, "launches": infos[0]["step_launches"],
                             "us_per_launch": 1e3 * dev_ms / max(infos[0]["step_launches"], 1),
                             "basis": "dense-method bytes of every fit's coordinate steps / CUDA-event time of the batch",
                             "peak_source": src}
        out[name] = r
        for hh in handles:
            hh.close()
        if plan is not None:
            cox.cox_set_chunk_plan(0)
    best = max(("batched_fp32c", "batched_fp64", "batched_incremental"), key=lambda k: out[k]["fits_per_s"])
    out["best"] = best
    out["fits_per_s"] = out[best]["fits_per_s"]
    if not sub:
        return {"metric": "fits/sec (256 CCD fits: 4 outcomes x 4 folds x 16 L1 weights)", "value": out["fits_per_s"],
                "unit": "fits/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic (seeded)",
                "config": {"workload": out["workload"]}, "batch": out}
    return out


# ---------------------------------------------------------------- config 5: serving
def run_serving(args, sub=False):
    """Poisson fit requests into the continuous-batching server (FP32C): its capacity under a
    burst, then a Poisson stream at 80 % of that capacity with p50 / p99 time-to-fit. The request
    pool is drawn from the full recipe (rows up to 1e7) on the device (synth_device); every
    arrival reuses a pool entry with its own penalty draw."""
    import torch
    from paper_2310_16238_gb300 import cox, synth_device
    prec = cox.COX_FP32C
    dev = torch.device("cuda", 0)
    reqs = synth.serving_stream(rate=args.rate, duration_s=120.0)
    t0 = time.perf_counter()
    pool = [(r, synth_device.request_data(r, dev)) for r in reqs[:args.pool]]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    rows = [int(d.n) for _, (d, _) in pool]
    nnz = [int(d.row_idx.numel()) for _, (d, _) in pool]
    rng = np.random.default_rng(7)

    def options(r, d):
        if r.penalty == synth.PEN_L1:
            return synth.CoxOptions(penalty=synth.PEN_L1, lam=float(np.exp(rng.uniform(-10, -6))) * d.n, tol=1e-8)
        return synth.CoxOptions(penalty=synth.PEN_L2, l2_var=float(np.exp(rng.uniform(-2, 1))), tol=1e-8)

    def drive(arrivals, timeout_s, fixed=None):
        """Submit pool[k % len(pool)] at arrivals[k] (options `fixed[k]`, else a fresh draw)."""
        lat, waits, fails, results = [], [], 0, {}
        with cox.Server(precision=prec) as srv:
            t_start = time.perf_counter()
            pending, k = {}, 0
            while k < len(arrivals) or pending:
                now = time.perf_counter() - t_start
                while k < len(arrivals) and arrivals[k] <= now:
                    r, (d, o) = pool[k % len(pool)]
                    pending[srv.submit(d, fixed[k] if fixed else options(r, d))] = k
                    k += 1
                for rid in list(pending):
                    try:
                        res = srv.poll(rid)
                    except cox.CoxError:
                        fails += 1
                        del pending[rid]
                        continue
                    if res is not None:
                        lat.append(res[1]["total_ms"])
                        waits.append(res[1]["wait_ms"])
                        results[pending[rid]] = res
                        del pending[rid]
                time.sleep(0.002)
                if now > timeout_s:
                    break
            elapsed = time.perf_counter() - t_start
            st = srv.stats()
        return np.array(lat), np.array(waits), elapsed, st, fails, results

    # capacity: every pool request submitted at t = 0
    burst_opts = [options(r, d) for r, (d, _) in pool]
    with ClockSampler(0) as clk_b:
        lat_b, _, el_b, _, _, res_b = drive([0.0] * len(pool), 900.0, fixed=burst_opts)
    capacity = len(lat_b) / el_b
    # the plain path on the same requests and options: one fit at a time, FP64 (AUTO engine)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk_p:
        t0 = time.perf_counter()
        plain = []
        for (r, (d, _)), o in zip(pool, burst_opts):
            with cox.Handle(d, o, precision=cox.COX_FP64) as h:
                plain.append(h.fit())
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - t0
    err, mism = 0.0, 0
    for k, (b32, i32) in res_b.items():
        b64, i64 = plain[k]
        if i32["sweeps"] != i64["sweeps"]:   # stopped one sweep apart: compare at the server's sweep
            mism += 1
            d = pool[k][1][0]
            o2 = dataclasses.replace(burst_opts[k], max_sweeps=int(i32["sweeps"]), tol=0.0)
            with cox.Handle(d, o2, precision=cox.COX_FP64) as h:
                b64, _ = h.fit()
        den = max(np.max(np.abs(b64)), 1e-12) if np.any(b64) else 1.0
        err = max(err, float(np.max(np.abs(np.asarray(b32) - b64)) / den))
    rate = 0.8 * capacity
    # a Poisson stream at 80 % of that capacity
    t, arr = 0.0, []
    r2 = np.random.default_rng(11)
    while True:
        t += r2.exponential(1.0 / rate)
        if t > args.duration:
            break
        arr.append(t)
    with ClockSampler(0) as clk:
        lat, waits, el, st, fails, _ = drive(arr, args.duration * 6)
    out = {"workload": "Poisson arrivals; requests rows logU[1e4,1e7], p logU[100,2e4], density logU[1e-4,1e-2], "
                       f"K U{{1..200}}, 50% counting-process, L1/L2 (a pool of {len(pool)} drawn on the device, no row cap)",
           "precision": "fp32c", "pool_rows": {"min": min(rows), "median": float(np.median(rows)), "max": max(rows)},
           "pool_nnz": {"median": float(np.median(nnz)), "max": max(nnz)}, "pool_generation_s": gen_s,
           "capacity_fits_per_s": capacity, "burst_requests": len(pool), "burst_s": el_b,
           "plain_fp64": {"fits_per_s": len(pool) / plain_s, "seconds": plain_s,
                          "engine": "AUTO per fit (one fit at a time, cox_create from the device arrays)",
                          "clocks": clk_p.summary()},
           "served_vs_plain": capacity / (len(pool) / plain_s),
           "max_rel_beta_err_vs_plain_fp64": err, "sweep_mismatches_vs_plain_fp64": mism,
           "sustainable_rate": rate, "offered_rate_config": args.rate,
           "stream": {"duration_s": args.duration, "requests": len(arr), "completed": len(lat), "failed": fails,
                      "fits_per_s": len(lat) / el,
                      "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                      "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                      "p50_wait_ms": float(np.percentile(waits, 50)) if len(waits) else None},
           "server": st, "clocks": clk.summary(), "clocks_burst": clk_b.summary()}
    del pool
    torch.cuda.empty_cache()
    if not sub:
        return {"metric": "fits/sec and p50/p99 time-to-fit (continuous-batching server)",
                "value": out["stream"]["fits_per_s"], "unit": "fits/s", "n_gpus": 1, "higher_is_better": True,
                "data": "synthetic (seeded request pool, drawn on the device)", "config": {"workload": out["workload"]},
                "serving": out}
    return out


# ---------------------------------------------------------------- other single workloads
def run_time_varying(args):
    """Counting-process fit (1e6 subjects, ~2.9e6 (start, stop] rows, p = 5000, K = 20, L2)."""
    import torch
    from paper_2310_16238_gb300 import cox
    data, opts = synth.time_varying(n_subj=int(1_000_000 * args.scale), p=5000, k=20)
    precision = cox.COX_FP32C if args.precision == "fp32c" else cox.COX_FP64
    engine = {"auto": cox.COX_ENGINE_AUTO, "stream": cox.COX_ENGINE_STREAM}[args.engine]
    stream = torch.cuda.Stream()
    times, infos = [], []
    with torch.cuda.stream(stream):
        h = cox.cox_create(data, opts, precision=precision, stream=stream.cuda_stream, engine=engine)
        for k in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            beta, info = cox.cox_fit(h)
            e1.record(stream)
            e1.synchronize()
            if k >= args.warmup:
                times.append(e0.elapsed_time(e1))
                infos.append(info)
        md = cox.cox_metadata(h)
        cox.cox_destroy(h)
    ms = float(np.mean(times))
    coords = float(np.mean([i["coord_updates"] for i in infos]))
    steps = float(np.mean([i["coord_updates"] + 1 for i in infos]))
    eng = ENGINE_NAMES.get(infos[-1]["engine"], "unknown")
    step_us = float(np.mean([i["sweep_ms"] for i in infos])) / steps * 1e3
    wname = f"time_varying subjects={int(1_000_000 * args.scale)} rows={data.n} p=5000 K=20 L2 var=0.1"
    s_e = 4 if precision == cox.COX_FP32C else 8
    roof = roofline_of(eng, data, beta, len(md["group_time"]), len(md["strata_start"]) - 1, s_e, step_us, wname,
                       args.precision)
    return {"metric": "coordinate updates/sec (CCD, counting-process Cox, one fit per step)",
            "value": coords / (ms * 1e-3), "unit": "coord_updates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(eng, s_e), "data": "synthetic (seeded)",
            "config": {"workload": wname, "precision": args.precision},
            "fit": {"sweeps": infos[-1]["sweeps"], "loglik": infos[-1]["loglik"], "step_us": step_us, "engine": eng},
            "roofline": roof}


def run_probe(args):
    """Small single-kernel cases for profiler captures (no graph, so every launch is a plain kernel
    launch a profiler can capture), timed with CUDA events:
      stream_fp32c / stream_fp64  cox_gradient (one evaluation launch per column) of the streaming
                                  kernels on time_varying(1e6 subjects, p=300, K=20)
      segscan                     cox_segscan on 2^24 doubles with 1,000 segments
      prep                        cox_create on the stratified sparse data of the default line
      incr / resident             one incremental- / resident-engine fit (1 sweep) of that data
      views                       a time-split view (cox_create_split) and a 5-fold CV path's subsets
      batch_fp32c                 one batched FP32C fit of the 256-fit batch workload (graph-replayed
                                  launches of the chunked kernel; the first sweep's hold every fit)"""
    import torch
    from paper_2310_16238_gb300 import cox
    what = args.probe
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"metric": "probe", "probe": what, "unit": "us"}
    with torch.cuda.stream(stream):
        if what in ("stream_fp32c", "stream_fp64"):
            d, o = synth.time_varying(n_subj=int(1_000_000 * args.scale), p=300, k=20)
            prec = cox.COX_FP32C if what == "stream_fp32c" else cox.COX_FP64
            beta = np.zeros(d.p)
            beta[::7] = 0.05

            def per_launch():
                with cox.Handle(d, o, precision=prec, engine=cox.COX_ENGINE_STREAM, stream=stream.cuda_stream) as h:
                    h.gradient(beta)
                    e0.record(stream)
                    h.gradient(beta)
                    e1.record(stream)
                    e1.synchronize()
                return 1e3 * e0.elapsed_time(e1) / d.p
            # the full pass first (the launches a profiler capture of this probe takes), then, FP32C,
            # the evaluation launches that read the tie groups' S0 kept from the first column's
            cox.cox_debug_set_cached_s0(False)
            out.update(value=per_launch(), what="us per evaluation launch (one column), full pass")
            cox.cox_debug_set_cached_s0(True)
            if prec == cox.COX_FP32C:
                out["cached_s0_us"] = per_launch()
        elif what == "segscan":
            n = 1 << 24
            g = torch.Generator(device="cuda").manual_seed(synth.SEED_BASE)
            a = torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
            f = torch.zeros(n, dtype=torch.uint8, device="cuda")
            f[torch.randint(0, n, (1000,), device="cuda", generator=g)] = 1
            cox.cox_segscan(a, f, stream=stream.cuda_stream)
            e0.record(stream)
            for _ in range(3):
                cox.cox_segscan(a, f, stream=stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            out.update(value=1e3 * e0.elapsed_time(e1) / 3, what="us per scan of 2^24 doubles")
        elif what == "resident":
            d, o, _ = headline_workload(args.scale)
            o = dataclasses.replace(o, max_sweeps=1)
            with cox.Handle(d, o, precision=cox.COX_FP64, engine=cox.COX_ENGINE_RESIDENT, stream=stream.cuda_stream) as h:
                e0.record(stream)
                beta, info = h.fit()
                e1.record(stream)
                e1.synchronize()
            out.update(value=1e3 * e0.elapsed_time(e1), what="us per 1-sweep fit",
                       engine=ENGINE_NAMES.get(info["engine"], "unknown"), steps=info["coord_updates"] + 1)
        elif what == "views":
            # the time-split view (a covariate split at two cut days) and a 5-fold CV path's row subsets
            d, o = synth.time_varying(n_subj=int(200_000 * args.scale), p=50, k=5)
            e0.record(stream)
            with cox.Handle.split(d, [90, 365], tvc_cols=(0, 1), opts=o, stream=stream.cuda_stream) as h:
                h.metadata()
            d2, o2 = synth.stratified_sparse(n=int(200_000 * args.scale), p=100, k=10, seed=synth.SEED_BASE + 7)
            fold = cox.make_folds(d2.n, 5, seed=7)
            cox.cox_cv_path(d2, fold, [1e-2 * d2.n, 1e-3 * d2.n], o2, n_folds=5, stream=stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            out.update(value=1e3 * e0.elapsed_time(e1), what="us for the split view and the CV path")
        elif what == "batch_fp32c":
            sets = synth.batch_views(n_total=int(1_000_000 * args.scale), n_lo=1e4 * args.scale,
                                     n_hi=1e6 * args.scale)
            handles = []
            for dd, ol in sets:
                base = cox.Handle(dd, ol[0], precision=cox.COX_FP32C, engine=cox.COX_ENGINE_STREAM,
                                  stream=stream.cuda_stream)
                handles.append(base)
                handles.extend(base.clone(oo) for oo in ol[1:])
            e0.record(stream)
            betas, infos = cox.batch_fit(handles)
            e1.record(stream)
            e1.synchronize()
            for hh in handles:
                hh.close()
            out.update(value=1e3 * e0.elapsed_time(e1) / max(infos[0]["step_launches"], 1),
                       what="us per batched launch (256 fits, averaged over the batch)",
                       launches=int(infos[0]["step_launches"]))
        elif what in ("prep", "incr"):
            d, o, _ = headline_workload(args.scale)
            if what == "prep":
                e0.record(stream)
                h = cox.Handle(d, o, precision=cox.COX_FP64, stream=stream.cuda_stream)
                e1.record(stream)
                e1.synchronize()
                h.close()
                out.update(value=1e3 * e0.elapsed_time(e1), what="us per cox_create (host inputs)")
            else:
                o = dataclasses.replace(o, max_sweeps=1)
                with cox.Handle(d, o, precision=cox.COX_FP64, stream=stream.cuda_stream) as h:
                    e0.record(stream)
                    beta, info = h.fit()
                    e1.record(stream)
                    e1.synchronize()
                out.update(value=1e3 * e0.elapsed_time(e1), what="us per 1-sweep fit",
                           engine=ENGINE_NAMES.get(info["engine"], "unknown"), steps=info["coord_updates"] + 1)
    return out


def run_cv(args):
    """10-fold cross-validation along an L1 path (the paper's tuning procedure, §3.2): a stratified
    sparse data set of 2e5 rows, p = 1000, 10 strata, 8 weights log-spaced from 1e-2 N down to
    1e-4 N; every weight's 10 training fits and the full-data fit run as one warm-started batch."""
    import torch
    from paper_2310_16238_gb300 import cox
    n = int(200_000 * args.scale)
    data, opts = synth.stratified_sparse(n=n, p=1000, k=10, n_support=30, event_frac=0.1, dens_lo=1e-3, dens_hi=5e-2,
                                         seed=synth.SEED_BASE + 7)
    K = 10
    fold = cox.make_folds(data.n, K, seed=7)
    path = list(np.logspace(np.log10(1e-2 * n), np.log10(1e-4 * n), 8))
    precision = cox.COX_FP32C if args.precision == "fp32c" else cox.COX_FP64
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    ddev = _device_copy(data, dev)
    dfold = torch.from_numpy(fold).to(dev)
    torch.cuda.synchronize()
    times, res = [], None
    with ClockSampler(0) as clk:
        with torch.cuda.stream(stream):
            for k in range(args.warmup + args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = cox.cox_cv_path(ddev, dfold, path, opts, n_folds=K, precision=precision,
                                      stream=stream.cuda_stream)
                e1.record(stream)
                e1.synchronize()
                if k >= args.warmup:
                    times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
    ms = float(np.mean(times))
    fits = len(path) * (K + 1)
    coords = sum(f["coord_updates"] for row in res["info"] for f in row)
    engines = sorted({ENGINE_NAMES.get(f["engine"], "unknown") for row in res["info"] for f in row})
    return {"metric": "fits/sec (10-fold cross-validated L1 path: 8 weights x (10 training + 1 full-data) fits, "
                      "warm-started batches)",
            "value": fits / (ms * 1e-3), "unit": "fits/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32x2+f64" if "incremental" in engines else ("f64" if precision == cox.COX_FP64 else "f32+f64"),
            "data": "synthetic (seeded)",
            "config": {"workload": f"stratified_sparse N={n} p=1000 K=10 strata, 10 folds, L1 path "
                                   f"{path[0]:.0f}..{path[-1]:.1f} (8 values)", "precision": args.precision},
            "cv": {"coord_updates_per_path": coords, "coord_updates_per_s": coords / (ms * 1e-3), "engines": engines,
                   "best": res["best"], "cvl": [float(v) for v in res["cvl"]],
                   "nonzero_at_best": int(np.count_nonzero(res["beta"][res["best"]]))},
            "clocks": clk.summary()}


def run_e1(args):
    """The paper's synthetic experiment shape (§3.1): N = 1e6, P = 2000, binary X at 5 % density,
    K equal strata (default 50,000), beta 20 % nonzero N(0, 1), L1 gamma = sqrt(2). One step = one
    full fit (cox_create from device-resident arrays + cox_fit + cox_destroy)."""
    import torch
    from paper_2310_16238_gb300 import cox
    n = int(1_000_000 * args.scale)
    K = args.strata if args.strata > 0 else 50_000
    data, opts = synth.synthetic_e1(n=n, p=2000, k=K)
    precision = cox.COX_FP32C if args.precision == "fp32c" else cox.COX_FP64
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    ddev = _device_copy(data, dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with ClockSampler(0) as clk:
        times, infos, beta, _ = _timed_fits(cox, ddev, opts, precision, stream, flush, args.steps, args.warmup)
    ms = float(np.mean(times))
    coords = float(np.mean([i["coord_updates"] for i in infos]))
    steps = float(np.mean([i["coord_updates"] + 1 for i in infos]))
    eng = ENGINE_NAMES.get(infos[-1]["engine"], "unknown")
    step_us = float(np.mean([i["sweep_ms"] for i in infos])) / steps * 1e3
    return {"metric": "seconds per fit (CCD to convergence, stratified L1 Cox; the paper's synthetic experiment shape)",
            "value": ms * 1e-3, "unit": "s/fit", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(eng, 8 if precision == cox.COX_FP64 else 4), "data": "synthetic (seeded)",
            "config": {"workload": f"synthetic_e1 N={n} p=2000 density 0.05 K={K} beta 20% N(0,1) L1 gamma=sqrt(2)",
                       "precision": args.precision},
            "fit": {"sweeps": infos[-1]["sweeps"], "coord_updates_per_s": coords / (ms * 1e-3),
                    "nonzero_beta": int(np.count_nonzero(beta)), "step_us": step_us, "engine": eng},
            "clocks": clk.summary()}


# ---------------------------------------------------------------- end to end from host buffers
def e2e(args, data, opts, stream):
    """Same metric through the public API with HOST buffers: the H2D copies of the inputs (inside
    cox_create, from pinned host memory) and the D2H of beta are inside the timed region."""
    import copy
    import torch
    from paper_2310_16238_gb300 import cox

    def pinned(a):   # a page-locked copy, made once outside the timed region
        return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    hdata = copy.copy(data)
    for k in ("stop", "start", "event", "stratum", "col_ptr", "row_idx", "val"):
        setattr(hdata, k, pinned(getattr(data, k)))
    h2d = sum(a.nbytes for a in (hdata.stop, hdata.start, hdata.event, hdata.stratum, hdata.col_ptr, hdata.row_idx,
                                 hdata.val) if a is not None)
    times, coords = [], []
    with torch.cuda.stream(stream):
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = cox.cox_create(hdata, opts, precision=cox.COX_FP64, stream=stream.cuda_stream)
            beta, info = cox.cox_fit(h)
            cox.cox_destroy(h)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            coords.append(info["coord_updates"])
    ms = float(np.mean(times))
    return {"value": float(np.mean(coords)) / (ms * 1e-3), "unit": "coord_updates/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(8 * data.p)}


# ---------------------------------------------------------------- the CPU oracle (baseline arm)
_CPU = {}


def _cpu_init(scale):
    """Worker set-up: the headline data (the same seed in every worker) and the built oracle."""
    import oracle
    oracle.build()
    data, opts, _ = headline_workload(scale)
    _CPU["data"], _CPU["opts"] = data, opts


def _cpu_run(ncoords):
    import oracle
    t0 = time.perf_counter()
    oracle.time_sample(_CPU["data"], _CPU["opts"], int(ncoords))
    return time.perf_counter() - t0


def usable_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


class OraclePool:
    """Independent oracle processes, one per core, each holding its own copy of the headline data:
    the fit replicated on every core (no shared state, no change to the oracle's arithmetic)."""

    def __init__(self, cores, scale):
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_cpu_init, initargs=(scale,))
        self.pool.map(_cpu_run, [1] * cores)          # every worker ready (data built, oracle loaded)

    def rate(self, ncoords):
        """Coordinate updates per second of all workers running `ncoords` each at once."""
        t0 = time.perf_counter()
        self.pool.map(_cpu_run, [ncoords] * self.cores, chunksize=1)
        return self.cores * ncoords / (time.perf_counter() - t0)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(scale, seconds):
    """The oracle as it stands on the host: one core, and one process per usable core."""
    import oracle
    oracle.build()
    data, opts, _ = headline_workload(scale)
    t0 = time.perf_counter()
    oracle.time_sample(data, opts, 2)
    per = (time.perf_counter() - t0) / 2
    n1 = max(2, int(0.5 * seconds / max(per, 1e-6)))
    t0 = time.perf_counter()
    oracle.time_sample(data, opts, n1)
    one = n1 / (time.perf_counter() - t0)
    cores = usable_cores()
    pool = OraclePool(cores, scale)
    try:
        allc = pool.rate(max(2, int(0.5 * seconds * one)))
    finally:
        pool.close()
    return {"value": allc, "unit": "coord_updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent oracle processes (one per usable core), each running "
                      f"{max(2, int(0.5 * seconds * one))} coordinate updates (Newton step + eta update) of the "
                      f"headline fit from beta = 0; FP64 C oracle",
            "single_core": {"value": one, "cores": 1, "sample": f"{n1} coordinate updates, one process"},
            "cpu": cpu_model()}


def _oracle_moving(q, scale):
    """Child process (run beside the GPU legs): the oracle's two-sweep iterate of the moving fit,
    then its fit of the small dense workload to convergence."""
    try:
        import oracle
        oracle.build()
        data, _, _ = headline_workload(scale)
        o = moving_options(data.n)
        b, info = oracle.fit(data, synth.CoxOptions(penalty=o.penalty, lam=o.lam, tol=0.0, max_sweeps=2), max_sweeps=2)
        d1, o1 = synth.plain_dense()
        b1, i1 = oracle.fit(d1, o1)
        q.put({"moving": (b, info["loglik"]), "plain": (b1, i1["loglik"], int(i1["sweeps"]))})
    except Exception as e:   # reported in the bench line, not fatal
        q.put(("error", repr(e)))


def run_reference(args, rank, world):
    if rank != 0:
        return None
    _, _, wname = headline_workload(args.scale)
    cores = usable_cores()
    pool = OraclePool(cores, args.scale)
    try:
        t0 = time.perf_counter()
        pool.rate(1)
        per = (time.perf_counter() - t0)
        budget = 150.0 / max(1, args.steps + args.warmup)
        ncoords = max(1, int(budget / max(per, 1e-6)))
        for _ in range(args.warmup):
            pool.rate(ncoords)
        rates = [pool.rate(ncoords) for _ in range(args.steps)]
    finally:
        pool.close()
    value = float(np.mean(rates))
    ms = 1e3 * cores * ncoords / value
    sample = (f"{cores} independent oracle processes (one per usable core), each running {ncoords} coordinate "
              f"updates of the same fit per step; FP64 C oracle")
    return {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "coord_updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "config": headline_config(wname),
            "parallelism": f"cpu oracle, {cores} processes on rank 0",
            "cpu_baseline": {"value": value, "unit": "coord_updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "coord_updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32c"])
    ap.add_argument("--engine", default="auto", choices=["auto", "stream"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of N (testing only)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="headline only (no moving / batch / serving sub-results)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--workload", default="default",
                    choices=["default", "time_varying", "cv", "e1", "batch", "serving", "probe"])
    ap.add_argument("--probe", default="stream_fp32c",
                    choices=["stream_fp32c", "stream_fp64", "segscan", "prep", "incr", "resident", "views", "batch_fp32c"],
                    help="probe workload: one small single-kernel case for a profiler capture")
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--duration", type=float, default=30.0)
    ap.add_argument("--pool", type=int, default=24)
    ap.add_argument("--strata", type=int, default=0, help="e1 workload: number of strata (default 50,000)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if args.workload != "default":
        fn = {"time_varying": run_time_varying, "cv": run_cv, "e1": run_e1, "batch": run_batch,
              "serving": run_serving, "probe": run_probe}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return
    # the oracle's iterate of the moving fit runs in its own process beside the GPU legs (started
    # before the first CUDA call)
    q = proc = None
    if rank == 0 and not args.no_sub:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        proc = ctx.Process(target=_oracle_moving, args=(q, args.scale), daemon=True)
        proc.start()
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res, (data, ddev, stream, flush, G, K) = run_headline(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_e2e:
            _, opts, _ = headline_workload(args.scale)
            res["e2e"] = e2e(args, data, opts, stream)
        if not args.no_sub:
            res["batch"] = run_batch(args, sub=True)
            if not args.no_serving:
                res["serving"] = run_serving(args, sub=True)
            res["counting_process"] = run_time_varying(argparse.Namespace(**{**vars(args), "steps": 2, "warmup": 1,
                                                                              "precision": "fp64", "engine": "auto"}))
            orc = None
            try:
                got = q.get(timeout=900)
                orc = got if isinstance(got, dict) else None
                if orc is None:
                    res["oracle_error"] = got[1]
            except Exception as e:
                res["oracle_error"] = repr(e)
            if proc is not None:
                proc.join(timeout=10)
            res["moving"] = run_moving(args, data, ddev, stream, flush, G, K, orc["moving"] if orc else None)
            res["plain"] = run_plain(args, stream, orc["plain"] if orc else None)
        if not args.no_cpu:
            res["cpu_baseline"] = cpu_baseline(args.scale, args.cpu_seconds)
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
