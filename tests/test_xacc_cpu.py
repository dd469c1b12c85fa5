"""CPU pins of the long accumulator that sums the Gram and norm terms in the
solver kernels (ccg_xacc.h, compiled here for the host from the same source).

What the mathematics fixes: the sum of products x_i y_i of doubles is a dyadic
rational, computed here exactly with Fractions.  The accumulator holds it
exactly within its window (terms 2^-150 below the largest lose their low
bits, at most n 2^-157 max|x_i y_i| in all) and returns the top 106 bits as
hi + lo, so

  |hi + lo - S| <= 2^-104 |S| + 2^-140 sum |x_i y_i| + 2^-1073   (n <= 2^17).

A single product of two doubles needs at most 106 bits, so hi + lo is then
the product itself; exact cancellation gives zero; Inf or NaN give NaN.  Both
variants (anchor moved up on the fly; anchor fixed by a pre-pass) must meet
the bound and agree bitwise when no term falls below the window.
"""
import ctypes
import math
import shutil
import subprocess
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def xdot(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    out = tmp_path_factory.mktemp("xacc") / "libxacc.so"
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", str(ROOT / "paper_1204_0069_gb300" / "csrc"),
                    str(ROOT / "tests" / "xacc_shim.cpp"), "-o", str(out)], check=True)
    lib = ctypes.CDLL(str(out))
    lib.xacc_dot.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_int,
                             ctypes.c_void_p]
    lib.xacc_dot_ldexp.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long,
                                   ctypes.c_void_p]

    def run(x, y, fixed):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        o = np.zeros(2)
        if fixed == "ldexp":
            lib.xacc_dot_ldexp(x.ctypes.data, y.ctypes.data, x.size, o.ctypes.data)
        else:
            lib.xacc_dot(x.ctypes.data, y.ctypes.data, x.size, int(fixed), o.ctypes.data)
        return float(o[0]), float(o[1])
    return run


def exact(x, y):
    return sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y)), Fraction(0))


def check_bound(hi, lo, x, y):
    S = exact(x, y)
    mag = sum((abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(x, y)), Fraction(0))
    err = abs(Fraction(hi) + Fraction(lo) - S)
    bound = Fraction(2) ** -104 * abs(S) + Fraction(2) ** -140 * mag + Fraction(2) ** -1073
    assert err <= bound, (float(err), float(bound))


def cases():
    rng = np.random.default_rng(11)
    out = []
    for t in range(60):
        n = int(rng.choice([1, 2, 7, 64, 500]))
        span = float(rng.choice([0.0, 5.0, 30.0, 200.0]))
        x = rng.standard_normal(n) * np.exp(rng.uniform(-span, span, n))
        y = rng.standard_normal(n) * np.exp(rng.uniform(-span, span, n))
        if t % 5 == 0:
            x, y = x * 1e-160, y * 1e-160     # products in the subnormal range
        if t % 7 == 0 and n > 1:
            y[: n // 2] = -x[: n // 2]        # partial cancellation
            x[: n // 2] = x[: n // 2]
        if t % 9 == 0:
            x[0] = 0.0
        out.append((x, y))
    return out


@pytest.mark.parametrize("fixed", [False, True])
def test_sums_within_the_bound(xdot, fixed):
    for x, y in cases():
        hi, lo = xdot(x, y, fixed)
        check_bound(hi, lo, x, y)


@pytest.mark.parametrize("fixed", [False, True])
def test_single_product_is_exact(xdot, fixed):
    rng = np.random.default_rng(3)
    for _ in range(200):
        a = float(rng.standard_normal() * math.exp(rng.uniform(-300, 300)))
        b = float(rng.standard_normal() * math.exp(rng.uniform(-300, 300)))
        hi, lo = xdot([a], [b], fixed)
        P = Fraction(a) * Fraction(b)
        if abs(P) > Fraction(2) ** -900:      # hi and lo both normal
            assert Fraction(hi) + Fraction(lo) == P
            # hi: the top 53 bits (truncated), lo: the rest
            assert abs(Fraction(hi)) <= abs(P) < abs(Fraction(hi)) + Fraction(math.ulp(hi))


@pytest.mark.parametrize("fixed", [False, True])
def test_exact_cancellation_zero_and_specials(xdot, fixed):
    x = np.array([1.5, -2.25e10, 3.0e-7, 7.0])
    y = np.array([2.0, 1.0e-3, 5.0, 0.0])
    xx = np.concatenate([x, x])
    yy = np.concatenate([y, -y])
    assert xdot(xx, yy, fixed) == (0.0, 0.0)
    assert xdot([0.0, 0.0], [1.0, -3.0], fixed) == (0.0, 0.0)
    for bad in (np.inf, -np.inf, np.nan):
        hi, _ = xdot([1.0, bad, 2.0], [1.0, 1.0, 1.0], fixed)
        assert math.isnan(hi)


@pytest.mark.parametrize("fixed", [False, True])
def test_headroom_of_many_largest_terms(xdot, fixed):
    n = 1 << 17
    x = np.full(n, 1.9999999999999998)     # largest significand
    y = np.full(n, -1.9999999999999998)
    hi, lo = xdot(x, y, fixed)
    S = n * Fraction(1.9999999999999998) ** 2
    assert Fraction(hi) + Fraction(lo) == -S


def test_both_variants_agree_inside_the_window(xdot):
    rng = np.random.default_rng(5)
    for _ in range(40):
        n = int(rng.integers(1, 300))
        x = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
        y = rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n))
        assert xdot(x, y, False) == xdot(x, y, True)


def test_bit_fields_match_the_ldexp_route(xdot):
    """hi and lo are assembled from their bit fields when normal; the same
    numbers written as (double) m * 2^s with ldexp must come out bit for bit,
    across the normal range, subnormal parts (rounded by ldexp on both
    routes), signed zeros and overflow to infinity."""
    rng = np.random.default_rng(21)
    sets = list(cases())
    for _ in range(200):
        n = int(rng.integers(1, 40))
        span = float(rng.choice([1.0, 40.0, 300.0]))
        scale = float(rng.choice([1.0, 1e-150, 1e-160, 1e-165, 1e150, 1e154]))
        x = rng.standard_normal(n) * np.exp(rng.uniform(-span, span, n)) * scale
        y = rng.standard_normal(n) * np.exp(rng.uniform(-span, span, n))
        sets.append((x, y))
    sets.append(([1e-160], [-1e-160]))            # lo part subnormal, negative
    sets.append(([1.7e308], [4.0]))               # overflows to infinity
    sets.append(([3.0, -3.0], [5.0, 5.0]))        # exact zero
    for x, y in sets:
        got = np.array(xdot(x, y, False))
        ref = np.array(xdot(x, y, "ldexp"))
        assert got.tobytes() == ref.tobytes() or (np.isnan(got[0]) and np.isnan(ref[0])), (got, ref)
