"""One fit sharded by stratum (shard.py + cox_shard_*) with the library's kernels on one GPU: the
shards are driven one after the other from one process (the collectives formed in place), so
no kernel waits on another. The sharded fit equals the oracle's fit of the whole data: 1e-9 in
beta, 1e-11 in the log-likelihood, on data where a stratum is split across three shards."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import shard, synth

pytestmark = pytest.mark.gpu
cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def _cases():
    one, o1 = synth.stratified_sparse(n=60000, p=10, k=1, n_support=4, event_frac=0.5, dens_lo=0.01, dens_hi=0.3,
                                      admin_days=2000, lam_per_n=2e-4, seed=31)
    many, o2 = synth.stratified_sparse(n=80000, p=8, k=9, n_support=4, event_frac=0.3, dens_lo=0.01, dens_hi=0.3,
                                       admin_days=1000, lam_per_n=2e-4, seed=32)
    o3 = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=0.5, tol=1e-10)
    tv, _ = synth.time_varying(n_subj=20000, p=8, k=5, density=0.05, event_frac=0.3, n_support=4, seed=33)
    return [("one_stratum_l1", one, o1, 3), ("zipf_strata_l2", many, o3, 3), ("zipf_strata_l1", many, o2, 4),
            ("counting_l2", tv, o3, 3)]


@pytest.mark.parametrize("name,data,opts,R", _cases(), ids=[c[0] for c in _cases()])
def test_sharded_fit_on_the_gpu_equals_the_oracle(name, data, opts, R):
    ob, oi = oracle.fit(data, opts)
    sh = shard.plan(data.stratum, data.stop, R, counting=data.start is not None, event=data.event)
    if name.startswith("one"):
        assert sh[0].continues_next and not sh[1].has_end   # the stratum spans every shard
    backends = [shard.GpuShard(shard.shard_data(data, s), opts, s) for s in sh]
    try:
        dxg = np.sum([b.local_dx() for b in backends], axis=0)   # the all-reduce of the ranks' delta'X
        for b in backends:
            b.setup(dxg)
        beta, info = shard.run_local(backends, sh, max_sweeps=oi["sweeps"])
    finally:
        for b in backends:
            b.close()
    assert info["sweeps"] == oi["sweeps"], (info, oi)
    assert np.max(np.abs(beta - ob)) <= 1e-9 * max(np.max(np.abs(ob)), 1e-300)
    assert abs(info["loglik"] - oi["loglik"]) <= 1e-11 * abs(oi["loglik"])
