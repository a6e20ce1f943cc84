"""Failure detection without a GPU fault: every device-side wait in the kernels (the look-back of
the streaming and segmented-scan kernels, the streaming kernel's pipeline stages, the record
exchange of the incremental kernel) gives up after a bounded number of SM clocks, and the call
then returns COX_E_TIMEOUT instead of hanging. Here the bound is set far too short for those
waits (cox_debug_set_wait_limit): no CTA skips a publish and nothing faults; the calls fail
cleanly, every CTA exits (the call returns), and the next calls on the same device, with the
default bound, succeed and give the right answer."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2310_16238_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
cox = pytest.importorskip("paper_2310_16238_gb300.cox")


@pytest.fixture(scope="module")
def data():
    # ~40 streaming tiles and a multi-CTA incremental plan: every call has waits between CTAs
    return synth.stratified_sparse(n=300_000, p=12, k=3, n_support=5, event_frac=0.1, dens_lo=0.01, dens_hi=0.2,
                                   admin_days=400, lam_per_n=1e-4, seed=77)


def _expect_timeout(fn):
    with pytest.raises(cox.CoxError) as e:
        fn()
    assert e.value.code == cox.COX_E_TIMEOUT, e.value


def test_short_wait_bound_fails_cleanly_then_calls_succeed(data):
    d, o = data
    rng = np.random.default_rng(3)
    n = 3_000_003
    a = torch.from_numpy(rng.integers(-9, 9, n).astype(np.float64)).cuda()
    f = torch.from_numpy((rng.random(n) < 1e-4).astype(np.uint8)).cuda()
    with cox.Handle(d, o, engine=cox.COX_ENGINE_STREAM) as hs, cox.Handle(d, o, engine=cox.COX_ENGINE_INCR) as hi:
        try:
            cox.cox_debug_set_wait_limit(1)   # one SM clock: any wait that does not succeed at once gives up
            _expect_timeout(hs.fit)
            _expect_timeout(hi.fit)
            _expect_timeout(lambda: cox.cox_segscan(a, f))
        finally:
            cox.cox_debug_set_wait_limit(0)
        torch.cuda.synchronize()
        # the same handles and device, default bound: clean results
        b1, i1 = hs.fit()
        b2, i2 = hi.fit()
    ob, oi = oracle.fit(d, o, max_sweeps=i1["sweeps"])
    for b, i in ((b1, i1), (b2, i2)):
        assert i["status"] >= 0 and i["sweeps"] == oi["sweeps"]
        assert np.max(np.abs(b - ob)) <= 1e-9 * max(np.max(np.abs(ob)), 1e-300)
    got = cox.cox_segscan(a, f).cpu().numpy()
    assert np.array_equal(got, oracle.segscan(a.cpu().numpy(), f.cpu().numpy()))
