"""The incremental kernel's double-word coordinate step (csrc/step_rule.cuh), built for the host,
against the oracle's FP64 step (§2.4: Newton step, trust region, L1 directional derivatives and
zero crossing, L2 prior) on random inputs that reach every branch. Computed steps agree to
double-word precision (1e-12 relative); a step clipped to the trust half-width, or one that stops an
L1 coefficient at zero, is the oracle's exactly (so the coefficient lands on an exact zero)."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2310_16238_gb300", "csrc")


@pytest.fixture(scope="module")
def driver():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "step_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "step_check.cpp"), "-o", exe], check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def _cases(rng, n):
    out = []
    for _ in range(n):
        pen = int(rng.choice([0, 1, 2]))
        g2 = float(np.exp(rng.uniform(-3, 5)))
        g1 = float(rng.normal(0, 1) * g2 * np.exp(rng.uniform(-4, 1)))
        b = 0.0 if rng.random() < 0.3 else float(rng.normal(0, 0.5))
        t = float(np.exp(rng.uniform(-4, 1)))
        lam = float(abs(g1) * np.exp(rng.uniform(-1, 1))) if rng.random() < 0.8 else 0.0
        var = float(np.exp(rng.uniform(-2, 2)))
        penalized = int(rng.random() < 0.9)
        if rng.random() < 0.1:
            g2 = -g2   # non-positive curvature: no step
        out.append((g1, g2, b, t, pen, lam, var, penalized))
    return out


def test_step_rule_matches_oracle(driver):
    rng = np.random.default_rng(11)
    cases = _cases(rng, 4000)
    lines = [f"{g1.hex()} {g2.hex()} {b.hex()} {t.hex()} {pen} {lam.hex()} {var.hex()} {pz}"
             for g1, g2, b, t, pen, lam, var, pz in cases]
    p = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    got = [float.fromhex(x) for x in p.stdout.split()]
    branches = {"zero": 0, "clip": 0, "cross": 0, "newton": 0}
    for (g1, g2, b, t, pen, lam, var, pz), s in zip(cases, got):
        ref, _ = oracle.step(g1, g2, b, t, pen, lam, var, pz)
        if ref == 0.0:
            branches["zero"] += 1
            assert s == 0.0, (g1, g2, b, t, pen, lam, var, pz, s)
            continue
        if pen == 1 and pz and b != 0.0 and ref == -b:
            branches["cross"] += 1
            assert s == -b and b + s == 0.0, (g1, g2, b, t, pen, lam, var, pz, s, ref)
        elif abs(ref) == t:
            branches["clip"] += 1
            assert s == ref, (g1, g2, b, t, pen, lam, var, pz, s, ref)
        else:
            branches["newton"] += 1
            assert abs(s - ref) <= 1e-12 * abs(ref), (g1, g2, b, t, pen, lam, var, pz, s, ref)
    assert all(v > 50 for v in branches.values()), branches
