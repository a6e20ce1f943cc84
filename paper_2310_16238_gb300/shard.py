"""One fit sharded by stratum across ranks (one process per GPU).

The stratified partial likelihood is a sum over strata (§2.1 eq. strat_l), and within a stratum
every risk-set sum is a suffix sum over its time-sorted rows (§2.6-§2.7). So the rows, sorted by
(stratum, stop), are cut into contiguous shards balanced by rows, one per rank:

* a cut falls between two distinct (stratum, stop) values, so a tie group and its risk-set head
  stay on one rank; where a stratum boundary lies close enough to the balanced cut, the cut
  moves there, and a stratum larger than the tolerance is split;
* a rank whose last stratum continues on the next rank needs, for its tie groups in that
  stratum, the sums of the continuation: one segmented suffix over the later ranks' head sums
  (each rank's sums from its first row to its first stratum end), gathered once per coordinate;
* the ranks' partial (G1, G2[, sum d log S0, beta'dX]) are summed once per coordinate, so every
  rank takes the same Newton step (§2.4) on its copy of beta.

Per coordinate: one all-gather of 4 doubles (skipped when no stratum is split) and one
all-reduce of 4 doubles. Counting-process data (start, stop] are cut at stratum boundaries only
(a row's exit from the risk set falls at its start time, anywhere in the stratum's time range).

This module holds the partition and the lock-step protocol; the per-rank arithmetic runs behind a
backend (`GpuShard`: the library's kernels through the C ABI) and the collectives behind a small
communicator over torch.distributed; `run_local` drives several shards from one process, with
the collectives done in place.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import synth


@dataclass
class Shard:
    rank: int
    lo: int                  # first row (in the sorted order)
    hi: int                  # one past the last row
    continues_prev: bool     # the first stratum started on an earlier rank
    continues_next: bool     # the last stratum continues on a later rank
    has_end: bool            # a stratum ends inside this shard (its first segment stops here)


def plan(stratum: Optional[np.ndarray], stop: np.ndarray, n_shards: int, counting: bool = False,
         tol: float = 0.1, event: Optional[np.ndarray] = None) -> List[Shard]:
    """Contiguous row ranges, one per rank, balanced by rows.

    Each cut is placed at the nearest stratum boundary within `tol` * (n / n_shards) rows of the
    balanced position; failing that (a large stratum), at the nearest row where the cut does not
    split a tie group (a block of equal (stratum, stop) holding an event; with `event` None, any
    block of equal (stratum, stop)). Counting-process data are cut at stratum boundaries only.
    Empty shards are allowed (more ranks than boundaries)."""
    n = int(stop.shape[0])
    s = np.zeros(n, np.int64) if stratum is None else np.asarray(stratum, np.int64)
    t = np.asarray(stop, np.int64)
    if n_shards <= 1 or n == 0:
        return [Shard(0, 0, n, False, False, n > 0)][:1] + [Shard(r, n, n, False, False, False) for r in range(1, n_shards)]
    stratum_start = np.flatnonzero(np.r_[True, s[1:] != s[:-1]])          # rows where a stratum begins
    new_block = np.r_[True, (s[1:] != s[:-1]) | (t[1:] != t[:-1])]
    if event is None:
        key_start = np.flatnonzero(new_block)
    else:   # inside a block without events a cut is allowed too
        bid = np.cumsum(new_block) - 1
        has_ev = np.bincount(bid, weights=np.asarray(event, np.float64), minlength=int(bid[-1]) + 1) > 0
        key_start = np.flatnonzero(new_block | ~has_ev[bid])
    cuts = [0]
    for r in range(1, n_shards):
        target = int(round(r * n / n_shards))
        i = np.searchsorted(stratum_start, target)
        cand = [stratum_start[k] for k in (i - 1, i) if 0 <= k < len(stratum_start)]
        best = min(cand, key=lambda c: abs(int(c) - target)) if cand else 0
        if counting or abs(int(best) - target) <= tol * n / n_shards:
            c = int(best)
        else:
            k = np.searchsorted(key_start, target)
            kc = [key_start[q] for q in (k - 1, k) if 0 <= q < len(key_start)]
            c = int(min(kc, key=lambda x: abs(int(x) - target)))
        cuts.append(max(c, cuts[-1]))
    cuts.append(n)
    out = []
    for r in range(n_shards):
        lo, hi = cuts[r], cuts[r + 1]
        cp = 0 < lo < n and lo < hi and s[lo] == s[lo - 1]
        cn = lo < hi < n and s[hi - 1] == s[hi]
        # a stratum ends inside the shard: some row before hi - 1 starts a new stratum, or the
        # shard's last row is a stratum's last row
        has_end = lo < hi and (bool(np.any(s[lo + 1:hi] != s[lo:hi - 1])) or not cn)
        out.append(Shard(r, lo, hi, bool(cp), bool(cn), bool(has_end)))
    return out


def shard_data(data: synth.CoxData, sh: Shard) -> synth.CoxData:
    """The shard's rows (re-indexed from 0) with every column restricted to them."""
    lo, hi = sh.lo, sh.hi
    cols, vals = [], []
    for j in range(data.p):
        a, b = int(data.col_ptr[j]), int(data.col_ptr[j + 1])
        r = data.row_idx[a:b]
        m = (r >= lo) & (r < hi)
        cols.append(r[m] - lo)
        if data.val is not None:
            vals.append(data.val[a:b][m])
    lens = np.array([len(c) for c in cols], np.int64)
    col_ptr = np.zeros(data.p + 1, np.int64)
    np.cumsum(lens, out=col_ptr[1:])
    row_idx = np.concatenate(cols).astype(np.int32) if len(cols) and lens.sum() else np.zeros(0, np.int32)
    return synth.CoxData(stop=data.stop[lo:hi].copy(), event=data.event[lo:hi].copy(),
                         stratum=None if data.stratum is None else data.stratum[lo:hi].copy(),
                         start=None if data.start is None else data.start[lo:hi].copy(),
                         col_ptr=col_ptr, row_idx=row_idx,
                         val=None if data.val is None else (np.concatenate(vals) if lens.sum() else np.zeros(0)),
                         p=data.p, recipe=f"{data.recipe} shard {sh.rank}")


def carry_for(rank: int, shards: Sequence[Shard], heads: np.ndarray) -> np.ndarray:
    """Sums of rank's last stratum on the later ranks: the head sums (rows [k] of `heads`, each a
    rank's sums from its first row to its first stratum end) of the ranks that continue it, up to
    and including the first that holds the stratum's end."""
    c = np.zeros(heads.shape[1])
    if not shards[rank].continues_next:
        return c
    for q in range(rank + 1, len(shards)):
        if not shards[q].continues_prev:
            break
        c += heads[q]
        if shards[q].has_end:
            break
    return c


class DistComm:
    """torch.distributed collectives (gloo on CPU tensors, NCCL on CUDA tensors)."""

    def __init__(self, device="cpu"):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.device = torch, dist, device
        self.n = dist.get_world_size()

    def allgather(self, vec):
        t = self.torch.as_tensor(np.asarray(vec, np.float64), device=self.device)
        out = [self.torch.empty_like(t) for _ in range(self.n)]
        self.dist.all_gather(out, t)
        return np.stack([o.cpu().numpy() for o in out])

    def allreduce(self, vec):
        t = self.torch.as_tensor(np.asarray(vec, np.float64), device=self.device).clone()
        self.dist.all_reduce(t)
        return t.cpu().numpy()


def run_rank(backend, shards: Sequence[Shard], rank: int, comm, max_sweeps: int = 1000):
    """The lock-step CCD of one rank; every rank calls it. `backend` holds the shard's state and
    arithmetic:
      head(j)                    applies the pending update of the previous step, then returns the
                                 shard's sums (S0, S1, S2, 0) from its first row to its first stratum end
      partial(j, carry, need_ll) the shard's (G1, G2, sum d log S0, beta'dX) for column j, with
                                 `carry` added to the sums of its last stratum
      step(j, tot, need_ll, sweep, max_sweeps) -> (state, loglik)
                                 the convergence test (when need_ll) and the coordinate step from
                                 the summed partials; state 0 = running, 1 = converged, 2 = sweeps
      beta()
    Returns (beta, info), identical on every rank."""
    split = any(s.continues_next for s in shards)
    p = backend.p
    sweep, updates, loglik = 0, 0, None
    while True:
        for j in range(p):
            need_ll = j == 0
            head = backend.head(j)
            carry = carry_for(rank, shards, comm.allgather(head)) if split else np.zeros_like(head)
            tot = comm.allreduce(backend.partial(j, carry, need_ll))
            state, ll = backend.step(j, tot, need_ll, sweep, max_sweeps)
            if need_ll:
                loglik = ll
            if state != 0:
                return backend.beta(), dict(sweeps=sweep, coord_updates=updates, loglik=loglik, converged=state == 1)
            updates += 1
        sweep += 1


def run_local(backends, shards: Sequence[Shard], max_sweeps: int = 1000):
    """The same lock-step protocol with every shard in this process: the gathered head sums and
    the summed partials are formed in place of the collectives."""
    split = any(s.continues_next for s in shards)
    p = backends[0].p
    sweep, updates, loglik = 0, 0, None
    while True:
        for j in range(p):
            need_ll = j == 0
            heads = np.stack([b.head(j) for b in backends])
            parts = [b.partial(j, carry_for(r, shards, heads) if split else np.zeros(heads.shape[1]), need_ll)
                     for r, b in enumerate(backends)]
            tot = np.sum(np.stack(parts), axis=0)
            res = [b.step(j, tot, need_ll, sweep, max_sweeps) for b in backends]
            state, ll = res[0]
            if need_ll:
                loglik = ll
            if state != 0:
                return backends[0].beta(), dict(sweeps=sweep, coord_updates=updates, loglik=loglik,
                                                converged=state == 1)
            updates += 1
        sweep += 1


class GpuShard:
    """A rank's shard on its GPU: a handle on the shard's rows (FP64, streaming kernel); head sums,
    partials and steps run in the library's kernels through the C ABI (cox_shard_*)."""

    def __init__(self, data_shard, opts, sh: Shard, stream=None):
        from . import cox
        self.cox, self.sh = cox, sh
        self.h = cox.Handle(data_shard, opts, precision=cox.COX_FP64, engine=cox.COX_ENGINE_STREAM, stream=stream)
        self.p = int(data_shard.p)

    def local_dx(self):
        """delta'X over the shard's rows (the ranks' sum is the whole fit's)."""
        return self.h.dx()

    def setup(self, dx_global):
        dxg = np.ascontiguousarray(dx_global, np.float64)
        self.cox._check(self.cox.lib().cox_shard_setup(self.h.h, dxg.ctypes.data, int(self.sh.continues_next)),
                        self.h.h)

    def head(self, j):
        out = np.zeros(4)
        self.cox._check(self.cox.lib().cox_shard_head(self.h.h, int(j), out.ctypes.data), self.h.h)
        return out

    def partial(self, j, carry, need_ll):
        c = np.ascontiguousarray(np.asarray(carry, np.float64)[:3])
        out = np.zeros(4)
        self.cox._check(self.cox.lib().cox_shard_partial(self.h.h, int(j), c.ctypes.data, int(need_ll), out.ctypes.data),
                        self.h.h)
        return out

    def step(self, j, tot, need_ll, sweep, max_sweeps):
        import ctypes as C
        t = np.ascontiguousarray(np.asarray(tot, np.float64)[:4])
        st, ll = C.c_int32(), C.c_double()
        self.cox._check(self.cox.lib().cox_shard_step(self.h.h, int(j), t.ctypes.data, int(need_ll), int(sweep),
                                                      int(max_sweeps), C.byref(st), C.byref(ll)), self.h.h)
        return int(st.value), (float(ll.value) if need_ll else None)

    def beta(self):
        b = np.zeros(max(self.p, 1))
        self.cox._check(self.cox.lib().cox_shard_beta(self.h.h, b.ctypes.data), self.h.h)
        return b[:self.p]

    def close(self):
        self.h.close()
