"""Small seeded test inputs built with the synthetic-data recipes (shared by CPU and GPU tests)."""
from __future__ import annotations

import numpy as np

from paper_2310_16238_gb300 import synth


def tiny_cases():
    """A handful of small data sets that stress ties, strata, sparse/dense X and start-stop rows."""
    out = []
    d, o = synth.plain_dense(n=60, p=4, seed=11)
    out.append(("dense_ties", d, o))
    d, o = synth.stratified_sparse(n=150, p=6, k=5, n_support=3, event_frac=0.3, dens_lo=0.05, dens_hi=0.5,
                                   admin_days=30, seed=12)
    out.append(("strata_sparse", d, o))
    d, o = synth.stratified_sparse(n=120, p=5, k=60, n_support=2, event_frac=0.5, dens_lo=0.1, dens_hi=0.6,
                                   admin_days=10, seed=13)
    out.append(("strata_half", d, o))       # K = n/2: size-2 strata
    d, o = synth.time_varying(n_subj=40, p=5, k=3, density=0.3, event_frac=0.5, n_support=3, seed=14)
    out.append(("start_stop", d, o))
    return out


def random_beta(p, scale=0.3, seed=0):
    return np.random.default_rng(seed).normal(0.0, scale, p)
