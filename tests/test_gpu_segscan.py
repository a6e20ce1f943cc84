"""The segmented-scan primitive (paper §2.6) on the GPU through the C ABI, against the
oracle's restatement of the operator and the paper's worked example."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
cox = pytest.importorskip("paper_2310_16238_gb300.cox")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "segscan_p704.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            out[k] = [float(x) for x in v]
    return out


def _run(a, f):
    ta = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    tf = torch.from_numpy(np.ascontiguousarray(f, dtype=np.uint8)).cuda()
    return cox.cox_segscan(ta, tf).cpu().numpy()


def test_paper_worked_example():
    g = _golden()
    assert _run(g["a"], g["f"]).tolist() == g["b"]


@pytest.mark.parametrize("n", [1, 7, 4095, 4096, 4097, 100_003, 3_000_001])
@pytest.mark.parametrize("head_p", [0.0, 1e-4, 0.05, 0.5, 1.0])
def test_integer_values_bit_exact(n, head_p):
    """Small integers sum exactly in FP64, so any association order gives the same bits."""
    rng = np.random.default_rng(n + int(head_p * 1000))
    a = rng.integers(-50, 50, n).astype(np.float64)
    f = (rng.random(n) < head_p).astype(np.uint8)
    assert np.array_equal(_run(a, f), oracle.segscan(a, f))


def test_real_values_and_heads_on_tile_boundaries():
    rng = np.random.default_rng(3)
    n = 4096 * 9 + 5
    a = rng.random(n)
    f = np.zeros(n, np.uint8)
    f[[0, 4095, 4096, 8192, 4096 * 5 - 1, n - 1]] = 1
    b, ref = _run(a, f), oracle.segscan(a, f)
    assert np.allclose(b, ref, rtol=1e-13, atol=0)


def test_rejects_host_pointers():
    a = np.zeros(4)
    f = np.zeros(4, np.uint8)
    rc = cox.lib().cox_segscan(a.ctypes.data, f.ctypes.data, 4, a.ctypes.data, None)
    assert rc == cox.COX_E_INVALID
