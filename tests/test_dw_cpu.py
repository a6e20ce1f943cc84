"""The double-word arithmetic of the incremental kernel (csrc/dw.cuh), built for the host and
checked in exact rational arithmetic: TwoSum and TwoProd are error-free, and the double-word sum,
products and quotient stay within the bounds published for these algorithms (Joldes, Muller and
Popescu, ACM TOMS 2017; u = 2^-24): sum 3u^2 + 13u^3, DW*FP 2u^2, DW*DW 5u^2, DW/DW
15u^2 + 56u^3, with normalized results (|l| <= ulp(h)/2)."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2310_16238_gb300", "csrc")
U = Fraction(1, 2 ** 24)
BOUND = {"add": 3 * U ** 2 + 13 * U ** 3, "addsame": 3 * U ** 2 + 13 * U ** 3, "mulf": 2 * U ** 2, "mul": 5 * U ** 2,
         "div": 15 * U ** 2 + 56 * U ** 3}


@pytest.fixture(scope="module")
def driver():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "dw_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, os.path.join(HERE, "dw_check.cpp"),
                    "-o", exe], check=True)
    yield exe
    shutil.rmtree(d, ignore_errors=True)


def _split(x):
    """Normalized double-word of a double: h = fl32(x), l = fl32(x - h)."""
    h = np.float32(x)
    return h, np.float32(x - float(h))


def _inputs(rng, n, same_sign=False):
    out = []
    for _ in range(n):
        e1, e2 = rng.integers(-30, 30, 2)
        a = rng.uniform(0.5, 1.0) * 2.0 ** e1 * rng.choice([-1.0, 1.0])
        b = rng.uniform(0.5, 1.0) * 2.0 ** e2 * rng.choice([-1.0, 1.0])
        if same_sign:
            b = abs(b) if a > 0 else -abs(b)
        elif rng.random() < 0.2:   # near-cancellation for the sum
            b = -a * (1.0 + rng.uniform(-1e-6, 1e-6))
        out.append((_split(a), _split(b)))
    return out


def _run(driver, lines):
    p = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return [tuple(float.fromhex(v) for v in ln.split()) for ln in p.stdout.strip().splitlines()]


def _fr(v):
    return Fraction(float(v))


def test_error_free_transforms(driver):
    rng = np.random.default_rng(5)
    cases = _inputs(rng, 400)
    lines = []
    for (xh, _), (yh, _) in cases:
        lines.append(f"twosum {float(xh).hex()} 0x0p+0 {float(yh).hex()} 0x0p+0")
        lines.append(f"twoprod {float(xh).hex()} 0x0p+0 {float(yh).hex()} 0x0p+0")
    res = _run(driver, lines)
    for k, ((xh, _), (yh, _)) in enumerate(cases):
        s, e = res[2 * k]
        assert _fr(s) + _fr(e) == _fr(xh) + _fr(yh)
        p, q = res[2 * k + 1]
        assert _fr(p) + _fr(q) == _fr(xh) * _fr(yh)


@pytest.mark.parametrize("op", ["add", "addsame", "mulf", "mul", "div"])
def test_double_word_ops_within_published_bounds(driver, op):
    rng = np.random.default_rng({"add": 1, "addsame": 5, "mulf": 2, "mul": 3, "div": 4}[op])
    cases = _inputs(rng, 600, same_sign=(op == "addsame"))
    lines = [f"{op} {float(a[0]).hex()} {float(a[1]).hex()} {float(b[0]).hex()} {float(b[1]).hex()}" for a, b in cases]
    res = _run(driver, lines)
    worst = Fraction(0)
    for (a, b), (rh, rl) in zip(cases, res):
        x = _fr(a[0]) + _fr(a[1])
        y = _fr(b[0]) + _fr(b[1]) if op != "mulf" else _fr(b[0])
        exact = {"add": x + y, "addsame": x + y, "mulf": x * y, "mul": x * y, "div": x / y}[op]
        got = _fr(rh) + _fr(rl)
        if exact == 0:
            assert got == 0
            continue
        rel = abs(got - exact) / abs(exact)
        worst = max(worst, rel)
        assert rel <= BOUND[op], (op, a, b, float(rel))
        # normalized: the low part is at most half an ulp of the high part
        if rh != 0.0:
            assert abs(_fr(rl)) <= abs(_fr(rh)) * U, (op, rh, rl)
    assert worst > 0   # the cases exercise rounding
