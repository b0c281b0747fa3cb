"""Double-double (compensated) arithmetic on numpy float64 arrays.

Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and the
product split of Dekker (Numer. Math. 18, 1971) -- numpy has no fused
multiply-add, so products are made exact with Veltkamp's 27-bit split.  A
double-double value is a pair (hi, lo) with |lo| <= ulp(hi)/2.  Used only to
evaluate residuals accurately for iterative refinement.
"""
import numpy as np

_SPLIT = 134217729.0  # 2^27 + 1


def two_sum(a, b):
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def dd_add(xh, xl, yh, yl):
    s, e = two_sum(xh, yh)
    e = e + (xl + yl)
    return two_sum(s, e)


def dd_add_d(xh, xl, y):
    s, e = two_sum(xh, y)
    e = e + xl
    return two_sum(s, e)


def dd_mul_d(xh, xl, b):
    p, e = two_prod(xh, b)
    e = e + xl * b
    return two_sum(p, e)


def dd_from_diff(a, b):
    """a - b as a double-double (exact)."""
    return two_sum(a, -b)
