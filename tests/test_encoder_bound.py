"""The certified encoder's error bound, checked in exact rational arithmetic.

The encoder computes y = fl(... fl(x_2 a_2 + fl(x_1 a_1 + 0)) ...) with one
rounding per fused multiply-add, and bounds |y - sum_i x_i a_i| by
gamma * (E + 8 ||x|| ||a||) + d 2^-148, where E adds 8 |s_c| at the start of
every chunk of 8 terms, gamma >= u / (1 - 8u), and every bound operation
rounds up.  Here each FP32 operation is replayed exactly (Fractions, round to
nearest even or upward), and the bound is checked against the exact dot
product on inputs chosen to stress it: cancellation, wide exponents,
subnormal products and zeros.  A coordinate whose interval holds no
breakpoint keeps the region of y, so a sound bound is what makes the codes
exact."""
import math
from fractions import Fraction

import numpy as np
import pytest

U = Fraction(1, 2 ** 24)
CH = 8


def _neighbours(f):
    f = np.float32(f)
    return [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]


def rn32(x):
    """x rounded to the nearest FP32, ties to even."""
    best = None
    for c in _neighbours(np.float32(float(x))):
        if not np.isfinite(c):
            continue
        e = abs(Fraction(float(c)) - x)
        key = (e, int(np.float32(c).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return np.float32(best[1])


def ru32(x):
    """The smallest FP32 >= x."""
    c = [v for v in _neighbours(np.float32(float(x))) if np.isfinite(v) and Fraction(float(v)) >= x]
    return np.float32(min(c, key=lambda v: Fraction(float(v))))


def sqrt_ru32(x):
    v = ru32(Fraction(math.sqrt(float(x))))
    while Fraction(float(v)) ** 2 < x:
        v = np.nextafter(v, np.float32(np.inf))
    while v > 0 and Fraction(float(np.nextafter(v, np.float32(0)))) ** 2 >= x:
        v = np.nextafter(v, np.float32(0))
    return v


def encoder_estimate_and_bound(x, a):
    d = len(x)
    F = lambda v: Fraction(float(v))  # noqa: E731
    s = np.float32(0.0)
    E = np.float32(0.0)
    for k in range(0, d, CH):
        E = ru32(8 * abs(F(s)) + F(E))
        for i in range(k, min(d, k + CH)):
            s = rn32(F(x[i]) * F(a[i]) + F(s))
    nx2 = np.float32(0.0)
    for v in x:
        nx2 = ru32(F(v) * F(v) + F(nx2))
    na2 = np.float32(0.0)
    for v in a:
        na2 = ru32(F(v) * F(v) + F(na2))
    nx, na = sqrt_ru32(F(nx2)), sqrt_ru32(F(na2))
    gam = ru32(U * (1 + 2 * CH * U) * Fraction(1000000001, 1000000000))
    tiny = np.float32(d * 2.0 ** -148)
    tot = ru32(8 * F(ru32(F(nx) * F(na))) + F(E))
    dlt = ru32(F(gam) * F(tot) + F(tiny))
    exact = sum(F(xi) * F(ai) for xi, ai in zip(x, a))
    return s, dlt, exact


def _cases():
    g = np.random.default_rng(11)
    out = []
    for d in (1, 7, 8, 9, 24, 64):
        out.append(("gauss", g.normal(size=d).astype(np.float32), g.normal(size=d).astype(np.float32)))
    # heavy cancellation: large alternating terms that nearly cancel
    x = np.tile(np.float32([1e6, -1e6]), 16) + g.normal(size=32).astype(np.float32)
    out.append(("cancel", x.astype(np.float32), np.ones(32, np.float32)))
    # wide exponents within a row
    x = (g.normal(size=48) * 2.0 ** g.integers(-30, 30, 48)).astype(np.float32)
    out.append(("wide", x, g.normal(size=48).astype(np.float32)))
    # subnormal products and zeros
    x = np.float32([1e-30, -3e-31, 0.0, 2e-29] * 5)
    a = np.float32([1e-10, 4e-9, 7.0, -1e-12] * 5)
    out.append(("tiny", x, a))
    # rounding errors of one sign: every product is 1 + ~1e-6, lost against
    # the growing partial sum at each step (the running |s_c| term is what
    # covers this; the Cauchy-Schwarz term alone would not)
    d = 1024
    out.append(("drift", np.full(d, np.float32(1 + 3 * 2.0 ** -23), np.float32),
                np.full(d, np.float32(1 + 5 * 2.0 ** -23), np.float32)))
    # integer-valued rows (SIFT-like) against Gaussian projections
    out.append(("ints", g.integers(0, 256, 128).astype(np.float32), g.normal(size=128).astype(np.float32)))
    return out


@pytest.mark.parametrize("name,x,a", _cases(), ids=[c[0] + str(len(c[1])) for c in _cases()])
def test_bound_covers_the_exact_dot_product(name, x, a):
    y, dlt, exact = encoder_estimate_and_bound(x, a)
    assert abs(Fraction(float(y)) - exact) <= Fraction(float(dlt)), (name, float(y), float(exact), float(dlt))


def test_bound_is_tight_enough_to_certify_most_coordinates():
    # typical rows: the bound is a small multiple of u * ||x|| ||a||
    g = np.random.default_rng(5)
    x = g.integers(0, 256, 128).astype(np.float32)
    a = g.normal(size=128).astype(np.float32)
    y, dlt, exact = encoder_estimate_and_bound(x, a)
    scale = float(np.linalg.norm(x.astype(np.float64)) * np.linalg.norm(a.astype(np.float64)))
    assert float(dlt) < 64 * 2.0 ** -24 * scale
