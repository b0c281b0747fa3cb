"""Pins of the double-double helpers of the oracle against exact rational
arithmetic: TwoSum and TwoProd are error-free transformations (Knuth;
Dekker), so hi + lo must equal the exact sum / product, and the compound
operations must stay within a few units of 2^-104 relative."""
from fractions import Fraction

import numpy as np

from oracle.dd import dd_add, dd_add_d, dd_from_diff, dd_mul_d, two_prod, two_sum


def _samples(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(-1.0, 1.0, n)
    expo = rng.integers(-30, 30, n)
    return np.ldexp(mant, expo)


def test_two_sum_and_two_prod_are_exact():
    a, b = _samples(400, 1), _samples(400, 2)
    s, e = two_sum(a, b)
    p, f = two_prod(a, b)
    for i in range(len(a)):
        assert Fraction(s[i]) + Fraction(e[i]) == Fraction(a[i]) + Fraction(b[i])
        assert Fraction(p[i]) + Fraction(f[i]) == Fraction(a[i]) * Fraction(b[i])
        assert s[i] == a[i] + b[i] and p[i] == a[i] * b[i]     # hi is the rounded result


def test_compound_operations_are_double_double_accurate():
    xh, yh, c = _samples(300, 3), _samples(300, 4), _samples(300, 5)
    xl = xh * np.ldexp(np.random.default_rng(6).uniform(-1, 1, 300), -54)
    yl = yh * np.ldexp(np.random.default_rng(7).uniform(-1, 1, 300), -54)
    sh, sl = dd_add(xh, xl, yh, yl)
    th, tl = dd_add_d(xh, xl, c)
    mh, ml = dd_mul_d(xh, xl, c)
    dh, dl = dd_from_diff(xh, c)
    for i in range(300):
        X, Y, C = Fraction(xh[i]) + Fraction(xl[i]), Fraction(yh[i]) + Fraction(yl[i]), Fraction(c[i])
        for hi, lo, exact, scale in (
                (sh[i], sl[i], X + Y, abs(X) + abs(Y)),
                (th[i], tl[i], X + C, abs(X) + abs(C)),
                (mh[i], ml[i], X * C, abs(X * C)),
                (dh[i], dl[i], Fraction(xh[i]) - C, 0)):
            err = abs(Fraction(hi) + Fraction(lo) - exact)
            assert err <= Fraction(2) ** -100 * scale, (i, float(err))
            assert abs(lo) <= abs(hi) * 2.0 ** -52     # normalised pair
