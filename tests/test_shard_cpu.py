"""Stratum sharding of one fit (paper_2310_16238_gb300/shard.py) on the CPU: the partition's
invariants, and the lock-step protocol -- one all-gather of head sums, one all-reduce of the
partials per coordinate, the same step on every rank -- run by two gloo ranks, with each rank's
arithmetic done by the oracle on its own rows (a stand-in for the rank's GPU). The sharded fit
must equal the oracle's fit of the whole data: 1e-9 in beta, 1e-11 in the log-likelihood."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2310_16238_gb300 import shard, synth


def _groups(d):
    """Tie groups of d in the oracle's order (stratum, then time): stratum and events of each."""
    s = np.zeros(d.n, np.int64) if d.stratum is None else d.stratum.astype(np.int64)
    ev = d.event.astype(bool)
    key = s[ev] * (1 << 32) + d.stop[ev].astype(np.int64)
    uk, cnt = np.unique(key, return_counts=True)
    return uk >> 32, cnt.astype(np.float64)


class OracleShard:
    """One rank's arithmetic on its rows, by the oracle: risk-set sums with the continuing
    stratum's carry added, ratios, and the oracle's step rule."""

    def __init__(self, data, sh, opts, dx_global):
        self.d = shard.shard_data(data, sh)
        self.sh, self.o, self.p = sh, opts, data.p
        self.b = np.zeros(self.p)
        self.tr = np.ones(self.p)
        self.dxg = dx_global
        self.dx = oracle.dX(self.d)
        self.gs, self.gd = _groups(self.d)
        s = np.zeros(self.d.n, np.int64) if self.d.stratum is None else self.d.stratum.astype(np.int64)
        self.last_stratum = s[-1] if self.d.n else -1
        ends = np.flatnonzero(np.r_[s[1:] != s[:-1], True])
        self.first_end = int(ends[0]) if len(ends) else -1
        self.obj_prev = None

    def _x(self, j):
        x = np.zeros(self.d.n)
        a, b = self.d.col_ptr[j], self.d.col_ptr[j + 1]
        x[self.d.row_idx[a:b]] = 1.0 if self.d.val is None else self.d.val[a:b]
        return x

    def head(self, j):
        e = np.exp(oracle.eta(self.d, self.b))[:self.first_end + 1]
        x = self._x(j)[:self.first_end + 1]
        return np.array([e.sum(), (x * e).sum(), (x * x * e).sum(), 0.0])

    def partial(self, j, carry, need_ll):
        S0, S1, S2 = oracle.risk_sums(self.d, self.b, j)
        if self.sh.continues_next:
            m = self.gs == self.last_stratum
            S0, S1, S2 = S0 + m * carry[0], S1 + m * carry[1], S2 + m * carry[2]
        r = S1 / S0
        out = [np.sum(self.gd * r), np.sum(self.gd * (S2 / S0 - r * r)), 0.0, 0.0]
        if need_ll:
            out[2] = np.sum(self.gd * np.log(S0))
            out[3] = float(self.b @ self.dx)
        return np.array(out)

    def _penalty(self):
        pen = np.ones(self.p, bool) if self.o.penalize is None else self.o.penalize.astype(bool)
        if self.o.penalty == synth.PEN_L1:
            return self.o.lam * np.sum(np.abs(self.b[pen]))
        if self.o.penalty == synth.PEN_L2:
            return np.sum(self.b[pen] ** 2) / (2.0 * self.o.l2_var)
        return 0.0

    def step(self, j, tot, need_ll, sweep, max_sweeps):
        ll = None
        if need_ll:
            ll = tot[3] - tot[2]
            obj = -ll + self._penalty()
            if sweep > 0 and abs(obj - self.obj_prev) <= self.o.tol * abs(obj):
                return 1, ll
            if sweep >= max_sweeps:
                return 2, ll
            self.obj_prev = obj
        pen = 1 if self.o.penalize is None else int(self.o.penalize[j])
        s, self.tr[j] = oracle.step(-self.dxg[j] + tot[0], tot[1], self.b[j], self.tr[j], self.o.penalty,
                                    self.o.lam, self.o.l2_var, pen)
        self.b[j] += s
        return 0, ll

    def beta(self):
        return self.b.copy()


def _cases():
    one, o1 = synth.stratified_sparse(n=600, p=6, k=1, n_support=3, event_frac=0.8, dens_lo=0.05, dens_hi=0.4,
                                      admin_days=400, lam_per_n=2e-3, seed=21)     # one stratum: split
    many, o2 = synth.stratified_sparse(n=900, p=5, k=7, n_support=3, event_frac=0.3, dens_lo=0.05, dens_hi=0.4,
                                       admin_days=60, lam_per_n=2e-3, seed=22)     # a Zipf head stratum: split
    o3 = synth.CoxOptions(penalty=synth.PEN_L2, l2_var=0.5, tol=1e-10)
    tv, _ = synth.time_varying(n_subj=300, p=5, k=4, density=0.2, event_frac=0.4, n_support=3, seed=23)
    return [("one_stratum_l1", one, o1), ("zipf_strata_l1", many, o2), ("zipf_strata_l2", many, o3),
            ("counting_l2", tv, o3)]


@pytest.mark.parametrize("name,data,opts", _cases(), ids=[c[0] for c in _cases()])
def test_plan_invariants(name, data, opts):
    for R in (2, 3, 5):
        sh = shard.plan(data.stratum, data.stop, R, counting=data.start is not None, event=data.event)
        assert [s.lo for s in sh][0] == 0 and sh[-1].hi == data.n
        assert all(a.hi == b.lo for a, b in zip(sh, sh[1:]))
        s = np.zeros(data.n, np.int64) if data.stratum is None else data.stratum.astype(np.int64)
        for a, b in zip(sh, sh[1:]):
            c = a.hi
            if 0 < c < data.n:
                # never inside a tie group (equal (stratum, stop) with an event); counting data only
                # at stratum ends
                same = (s == s[c]) & (data.stop == data.stop[c])
                assert (s[c] != s[c - 1]) or (data.stop[c] != data.stop[c - 1]) or not np.any(data.event[same])
                if data.start is not None:
                    assert s[c] != s[c - 1]
                assert a.continues_next == b.continues_prev == (s[c] == s[c - 1])
        sizes = [x.hi - x.lo for x in sh]
        if data.stratum is None or len(np.unique(data.stratum)) == 1:
            # balanced, up to the largest tie group (a cut never splits one)
            key = data.stop.astype(np.int64)
            _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
            has_ev = np.bincount(inv, weights=data.event.astype(float)) > 0
            biggest = int(np.max(cnt[has_ev])) if np.any(has_ev) else 0
            assert max(sizes) - min(sizes) <= 0.2 * data.n / R + 2 * biggest


@pytest.mark.parametrize("name,data,opts", _cases(), ids=[c[0] for c in _cases()])
def test_local_sharded_fit_equals_the_oracle(name, data, opts):
    ob, oi = oracle.fit(data, opts)
    sh = shard.plan(data.stratum, data.stop, 3, counting=data.start is not None, event=data.event)
    dxg = oracle.dX(data)
    backends = [OracleShard(data, s, opts, dxg) for s in sh]
    if name.startswith("one"):
        assert sh[0].continues_next and sh[1].continues_prev and not sh[1].has_end   # a stratum over 3 ranks
    b, info = shard.run_local(backends, sh, max_sweeps=oi["sweeps"])
    assert info["sweeps"] == oi["sweeps"]
    assert np.max(np.abs(b - ob)) <= 1e-9 * max(np.max(np.abs(ob)), 1e-300)
    assert abs(info["loglik"] - oi["loglik"]) <= 1e-11 * abs(oi["loglik"])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    name, data, opts = _cases()[case]
    sh = shard.plan(data.stratum, data.stop, world, counting=data.start is not None, event=data.event)
    be = OracleShard(data, sh[rank], opts, oracle.dX(data))
    b, info = shard.run_rank(be, sh, rank, shard.DistComm("cpu"))
    out[rank] = (b, info["loglik"], info["sweeps"])
    dist.destroy_process_group()


@pytest.mark.parametrize("case", [0, 1])
def test_two_gloo_ranks_fit_equals_the_oracle(case):
    name, data, opts = _cases()[case]
    ob, oi = oracle.fit(data, opts)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, _free_port(), case, out), nprocs=2, join=True)
        res = dict(out)
    (b0, l0, s0), (b1, l1, s1) = res[0], res[1]
    assert np.array_equal(b0, b1) and l0 == l1 and s0 == s1 == oi["sweeps"]   # every rank took the same steps
    assert np.max(np.abs(b0 - ob)) <= 1e-9 * max(np.max(np.abs(ob)), 1e-300)
    assert abs(l0 - oi["loglik"]) <= 1e-11 * abs(oi["loglik"])
