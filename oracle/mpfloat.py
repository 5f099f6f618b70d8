"""Radix-2^32 truncating floating point, n limbs -- the oracle's number format.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.1 of the paper stores every entry as an integer over 2^K and truncates
after each LDL^T.  Here the same "compute exactly, then truncate" rule is
applied to a floating format: a number is a pair ``(m, e)`` with value
m * 2**(32*e); ``m`` is a Python int whose magnitude has exactly n 32-bit
limbs (the top limb is non-zero) unless the value is zero, which is ``(0, 0)``.

``rnd(v, e)`` is the single rounding used everywhere: it takes an exact value
v * 2**(32*e) (v any Python int) and keeps the top n limbs of |v|, dropping
the rest (truncation of the magnitude toward zero).  Every primitive below
forms its exact result with Python's unbounded integers and calls ``rnd``
once, so each result is the exact value truncated to n limbs.
"""
from fractions import Fraction

LIMB = 32
ZERO = (0, 0)


def rnd(v, e, n):
    """Truncate the exact value v * 2**(32*e) to n limbs (toward zero)."""
    if v == 0:
        return ZERO
    neg = v < 0
    a = -v if neg else v
    limbs = (a.bit_length() + LIMB - 1) // LIMB
    if limbs > n:
        a >>= LIMB * (limbs - n)
        e += limbs - n
    elif limbs < n:
        a <<= LIMB * (n - limbs)
        e -= n - limbs
    return (-a if neg else a, e)


def from_int(v, n):
    """An exact integer truncated into the format."""
    return rnd(v, 0, n)


def from_fraction(q, n):
    """trunc_n of an exact rational q (magnitude floored to n limbs)."""
    q = Fraction(q)
    if q == 0:
        return ZERO
    neg = q < 0
    num, den = abs(q.numerator), q.denominator
    # find e such that floor(|q| / 2^(32 e)) has exactly n limbs
    e = (num.bit_length() - den.bit_length()) // LIMB - n
    while True:
        if e >= 0:
            m = num // (den << (LIMB * e))
        else:
            m = (num << (LIMB * -e)) // den
        limbs = (m.bit_length() + LIMB - 1) // LIMB
        if limbs > n:
            e += 1
        elif limbs < n:
            e -= 1
        else:
            return (-m if neg else m, e)


def to_fraction(x):
    m, e = x
    return Fraction(m) * Fraction(2) ** (LIMB * e)


def neg(x):
    return (-x[0], x[1])


def add(a, b, n):
    """trunc_n(a + b)."""
    (am, ae), (bm, be) = a, b
    if am == 0:
        return rnd(bm, be, n)
    if bm == 0:
        return rnd(am, ae, n)
    e = min(ae, be)
    return rnd((am << (LIMB * (ae - e))) + (bm << (LIMB * (be - e))), e, n)


def sub(a, b, n):
    return add(a, neg(b), n)


def mul(x, y, n):
    """trunc_n(x * y)."""
    return rnd(x[0] * y[0], x[1] + y[1], n)


def fused(a, x, y, n):
    """trunc_n(a - x*y) with the product x*y taken exactly (one rounding).

    This is the update of Algorithm 1, A_j[k] = A_j[k] - A_i[j]*B_i[k]
    (Sec. 4.3), and of Algorithm 4, A[j][k] = A[j][k] - f*A[i][k] (Sec. 4.4).
    """
    (am, ae), (xm, xe), (ym, ye) = a, x, y
    pm, pe = xm * ym, xe + ye
    if pm == 0:
        return rnd(am, ae, n)
    if am == 0:
        return rnd(-pm, pe, n)
    e = min(ae, pe)
    return rnd((am << (LIMB * (ae - e))) - (pm << (LIMB * (pe - e))), e, n)


def div(a, d, n):
    """trunc_n(a / d): the exact quotient with its magnitude floored to n limbs.

    The paper divides every entry of the pivot column by the pivot
    (B_i[j] = A_i[j]/A_i[i], Algorithm 1, Sec. 4.3).
    """
    (am, ae), (dm, de) = a, d
    if dm == 0:
        raise ZeroDivisionError("division by a zero pivot")
    if am == 0:
        return ZERO
    A, D = abs(am), abs(dm)
    # A, D both have n limbs, so floor(A * 2^(32n) / D) has n or n+1 limbs
    q = (A << (LIMB * n)) // D
    e = ae - de - n
    if q >> (LIMB * n):
        q = (A << (LIMB * (n - 1))) // D
        e += 1
    return (-q if (am < 0) != (dm < 0) else q, e)


def is_normal(x, n):
    """Format invariant: zero is (0, 0); otherwise |m| has exactly n limbs."""
    m, e = x
    if m == 0:
        return e == 0
    return (abs(m).bit_length() + LIMB - 1) // LIMB == n


def ulp(x):
    """Weight of the lowest limb of x (x != 0)."""
    return Fraction(2) ** (LIMB * x[1])


def limbs_of(x, n):
    """(sign, exp, [n little-endian 32-bit limbs]) -- the interchange layout."""
    m, e = x
    a = abs(m)
    return (1 if m < 0 else 0, e, [(a >> (LIMB * i)) & 0xFFFFFFFF for i in range(n)])


def from_limbs(sign, exp, limbs):
    a = 0
    for i, w in enumerate(limbs):
        a |= int(w) << (LIMB * i)
    if a == 0:
        return ZERO
    return (-a if sign else a, int(exp))


def to_mpf(x, mp):
    """Exact conversion to an mpmath mpf (the caller sets mp.prec >= 32 n)."""
    m, e = x
    return mp.ldexp(mp.mpf(m), LIMB * e)


def to_float(x):
    m, e = x
    if m == 0:
        return 0.0
    # keep 64 significant bits, then scale (avoids int->float overflow)
    sh = max(0, abs(m).bit_length() - 64)
    from math import ldexp
    return ldexp(float(m >> sh if m > 0 else -((-m) >> sh)), sh + LIMB * e)
