"""The float-float arithmetic of the FP32-mixed cost (csrc/ff.cuh), built as
plain C++ on the host with the same IEEE operations as the device build, and
checked against exact rational arithmetic (fractions.Fraction).

With u = 2^-24 (the unit roundoff of binary32) the pins are:
- the sum of two floats (Knuth's two-sum) and, for |a| >= |b|, Dekker's
  fast two-sum are error-free: hi = fl(a + b) and hi + lo = a + b exactly;
- a double splits as hi = fl32(d) with |d - (hi + lo)| <= u^2 |d|;
- the product: p = fl(xh yh) and its exact error (one FMA), the cross terms
  xh yl + xl yh rounded twice (<= 2u^2 |xy|), their sum with the error rounded
  once (<= 3u^2 |xy|), xl yl dropped (<= u^2 |xy|): |error| <= 8u^2 |xy|;
- the sum (Dekker's sloppy addition): the two heads summed exactly, the tails
  with two roundings and the renormalisation: |error| <= 4u^2 (|x| + |y|),
  a bound relative to |x| + |y| that holds under cancellation, where no bound
  relative to |x + y| does;
- the reciprocal after one Newton step: the float reciprocal has
  |1 - a x0| <= 2u + u^2, Newton squares that (<= 4u^2 + ...), and the step's
  float-float product and sum add at most 9u^2: |1 - a r| <= 16u^2;
- every result is normalised: |lo| <= u |hi|.
A dropped error term, a swapped operand in a two-sum or a contracted product
breaks the exactness checks by far more than these bounds."""
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U = Fr(1, 2**24)


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("ff") / "ff_host_check")
    cmd = [gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-Wall", "-I",
           os.path.join(ROOT, "paper_2112_01349_gb300", "csrc"), os.path.join(ROOT, "tests", "ff_host_check.cpp"),
           "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _run(exe, lines):
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = [tuple(float.fromhex(v) for v in ln.split()) for ln in r.stdout.strip().splitlines()]
    assert len(out) == len(lines)
    return out


def _h(v):
    return float(v).hex()


def _f32(rng, n, lo=-20, hi=20):
    """Floats with random signs, 24-bit mantissas and exponents in [lo, hi]."""
    m = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    return (m * np.exp2(rng.integers(lo, hi + 1, n))).astype(np.float32)


def _ff(rng, n, lo=-20, hi=20):
    """Normalised float-float values: hi = fl32(d), lo = fl32(d - hi)."""
    d = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n) * np.exp2(rng.integers(lo, hi + 1, n))
    h = d.astype(np.float32)
    return np.stack([h, (d - h.astype(np.float64)).astype(np.float32)], axis=1)


def _val(pair):
    return Fr(float(pair[0])) + Fr(float(pair[1]))


def _normalised(res):
    for h, l in res:
        assert abs(Fr(l)) <= U * abs(Fr(h)), (h, l)


def test_two_sums_are_error_free(exe):
    rng = np.random.default_rng(1)
    a, b = _f32(rng, 3000), _f32(rng, 3000)
    b[:500] = -a[:500]                                     # exact cancellation
    b[500:1000] = -a[500:1000] * np.float32(1 + 2**-20)    # near cancellation
    b[1000:1200] = 0.0
    res = _run(exe, [f"two_sum {_h(x)} {_h(y)}" for x, y in zip(a, b)])
    for x, y, (h, l) in zip(a, b, res):
        assert h == float(np.float32(x) + np.float32(y))
        assert Fr(h) + Fr(l) == Fr(float(x)) + Fr(float(y))
    big = np.where(np.abs(a) >= np.abs(b), a, b)
    small = np.where(np.abs(a) >= np.abs(b), b, a)
    res = _run(exe, [f"fast_two_sum {_h(x)} {_h(y)}" for x, y in zip(big, small)])
    for x, y, (h, l) in zip(big, small, res):
        assert Fr(h) + Fr(l) == Fr(float(x)) + Fr(float(y))


def test_split_of_a_double(exe):
    rng = np.random.default_rng(2)
    d = rng.normal(size=2000) * np.exp2(rng.integers(-30, 30, 2000))
    res = _run(exe, [f"from_d {_h(v)}" for v in d])
    for v, (h, l) in zip(d, res):
        assert h == float(np.float32(v))
        assert abs(Fr(float(v)) - Fr(h) - Fr(l)) <= U * U * abs(Fr(float(v)))
    _normalised(res)


def test_product_error_bound(exe):
    rng = np.random.default_rng(3)
    x, y = _ff(rng, 3000), _ff(rng, 3000)
    res = _run(exe, [f"mul {_h(a[0])} {_h(a[1])} {_h(b[0])} {_h(b[1])}" for a, b in zip(x, y)])
    worst = Fr(0)
    for a, b, r in zip(x, y, res):
        exact = _val(a) * _val(b)
        err = abs(_val(r) - exact) / abs(exact)
        worst = max(worst, err)
    assert worst <= 8 * U * U, float(worst / (U * U))
    _normalised(res)


@pytest.mark.parametrize("op", ["add", "sub"])
def test_sum_error_bound(exe, op):
    rng = np.random.default_rng(4 if op == "add" else 5)
    x, y = _ff(rng, 3000), _ff(rng, 3000)
    sgn = 1 if op == "add" else -1
    # cancellation: the heads of x and -y (add) or x and y (sub) equal or a
    # few ulps apart, with tails of their own, still normalised
    rho = rng.uniform(-1.0, 1.0, 1200).astype(np.float32)
    y[:600, 0] = -sgn * x[:600, 0]
    y[600:1200, 0] = -sgn * x[600:1200, 0] * np.float32(1 + 2**-22)
    y[:1200, 1] = (x[:1200, 1] * rho).astype(np.float32)
    y[1200:1500] = -sgn * x[1200:1500]                      # exact zero result
    for v in (x, y):
        assert all(abs(Fr(float(l))) <= U * abs(Fr(float(h))) for h, l in v)
    res = _run(exe, [f"{op} {_h(a[0])} {_h(a[1])} {_h(b[0])} {_h(b[1])}" for a, b in zip(x, y)])
    worst = Fr(0)
    for a, b, r in zip(x, y, res):
        exact = _val(a) + sgn * _val(b)
        scale = abs(_val(a)) + abs(_val(b))
        worst = max(worst, abs(_val(r) - exact) / scale)
    assert worst <= 4 * U * U, float(worst / (U * U))
    _normalised(res)


def test_reciprocal_error_bound(exe):
    rng = np.random.default_rng(6)
    a = _ff(rng, 3000, -40, 40)
    res = _run(exe, [f"rcp {_h(v[0])} {_h(v[1])}" for v in a])
    worst = max(abs(1 - _val(v) * _val(r)) for v, r in zip(a, res))
    assert worst <= 16 * U * U, float(worst / (U * U))
    _normalised(res)
