"""cox_segscan_noalloc: the entry point for callers that cannot allocate device memory while
they run (a host whose own pool must own every device byte, a real-time loop, a fixed memory
budget). It must give the same result as cox_segscan, call after call, although all calls
share one static scratch array that keeps the previous call's contents, and it must not ask
the library allocator for memory.

This file is named to be collected last, so that a run stopping at the first failure has
already run every other test."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
cox = pytest.importorskip("paper_2310_16238_gb300.cox")


def _call(fn, a, f):
    out = torch.full_like(a, float("nan"))
    rc = fn(a.data_ptr(), f.data_ptr(), C.c_int64(a.numel()), out.data_ptr(), None)
    assert rc == cox.COX_OK, cox.lib().cox_last_error(None).decode()
    return out.cpu().numpy()


class _CountingAllocator:
    """Library allocator that counts calls and forwards to torch's caching allocator."""

    def __init__(self):
        self.allocs = 0
        self.frees = 0

        def alloc(nbytes, ctx):
            self.allocs += 1
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))

        def free(ptr, nbytes, ctx):
            self.frees += 1
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._a, self._f = cox._ALLOC(alloc), cox._FREE(free)

    def __enter__(self):
        cox.lib().cox_set_allocator(self._a, self._f, None)
        return self

    def __exit__(self, *exc):
        cox.lib().cox_set_allocator(cox._ALLOC(), cox._FREE(), None)   # back to cudaMalloc / cudaFree
        cox._install_torch_allocator(cox.lib())                         # then to torch, as the binding sets it


@pytest.mark.parametrize("n,integer", [(4096 * 37 + 11, True), (1_000_003, False), (16_777_216, True)])
def test_noalloc_matches_allocating_entry_point_on_two_calls(n, integer):
    L = cox.lib()
    rng = np.random.default_rng(n)
    for call in range(2):
        a_np = rng.integers(-9, 9, n).astype(np.float64) if integer else rng.random(n)
        f_np = (rng.random(n) < (0.001 if call == 0 else 0.2)).astype(np.uint8)
        a = torch.from_numpy(a_np).cuda()
        f = torch.from_numpy(f_np).cuda()
        ref = _call(L.cox_segscan, a, f)
        with _CountingAllocator() as counter:
            got = _call(L.cox_segscan_noalloc, a, f)
        assert counter.allocs == 0 and counter.frees == 0, (counter.allocs, counter.frees)
        if integer:
            assert np.array_equal(got, ref), call      # exact sums: bit-exact, as in the other tests
        else:
            assert np.allclose(got, ref, rtol=1e-13, atol=0), call
        if integer and n == 16_777_216:
            # at the size limit the static path also equals the oracle's scan (integer sums are exact)
            assert np.array_equal(got, oracle.segscan(a_np, f_np)), call


def test_noalloc_rejects_sizes_beyond_its_static_limit():
    L = cox.lib()
    n = 16_777_216 + 1
    a = torch.zeros(n, dtype=torch.float64, device="cuda")
    f = torch.zeros(n, dtype=torch.uint8, device="cuda")
    out = torch.empty_like(a)
    rc = L.cox_segscan_noalloc(a.data_ptr(), f.data_ptr(), C.c_int64(n), out.data_ptr(), None)
    assert rc == cox.COX_E_INVALID
    assert b"16,777,216" in L.cox_last_error(None)
