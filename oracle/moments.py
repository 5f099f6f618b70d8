"""Moments mu_j = Gamma((j+1)/beta) / beta of w(x) = exp(-x^beta) on [0, inf).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2, eqs. "weight" and "moments".  For beta = 1/m (m a positive integer)
the moments are integers: mu_j = m * Gamma(m (j+1)) = m * (m(j+1) - 1)!, so
beta = 1/2 gives mu_j = 2 (2j+1)! and beta = 1 gives mu_j = j!.  Those are
formed exactly and truncated once.  For any other rational beta the value is
transcendental; it is evaluated with mpmath at 32 n + 128 bits and then
truncated (``gamma_moments``).
"""
from fractions import Fraction
from math import factorial

from . import mpfloat as F


def moment_exact(j, m):
    """mu_j for beta = 1/m as an exact integer."""
    return m * factorial(m * (j + 1) - 1)


def moments(beta, N, n):
    """[mu_0 .. mu_{2N-2}] truncated to n limbs; beta a Fraction or (num, den)."""
    beta = Fraction(*beta) if isinstance(beta, tuple) else Fraction(beta)
    if beta.numerator == 1:
        m = beta.denominator
        return [F.from_int(moment_exact(j, m), n) for j in range(2 * N - 1)]
    return gamma_moments(beta, N, n)


def gamma_moments(beta, N, n, extra_bits=128):
    """mu_j = Gamma((j+1)/beta)/beta via mpmath, then truncated to n limbs.

    beta may be any positive rational (or an mpmath number when the caller
    wants a perturbed beta for a finite difference).
    """
    import mpmath as mpm
    out = []
    with mpm.workprec(32 * n + extra_bits):
        b = mpm.mpf(beta.numerator) / beta.denominator if isinstance(beta, Fraction) else mpm.mpf(beta)
        for j in range(2 * N - 1):
            v = mpm.gamma((j + 1) / b) / b
            out.append(mpf_to_format(v, n, mpm))
    return out


def mpf_to_format(v, n, mpm):
    """Truncate an mpmath value (treated as exact) to n limbs."""
    if v == 0:
        return F.ZERO
    man, exp = mpm.mpf(v).man_exp
    # value = man * 2^exp exactly; express at a limb-aligned exponent
    e32, r = divmod(exp, 32)
    return F.rnd(int(man) << r, e32, n)


# --- rational beta = a/b through a-1 constants --------------------------------
# (j+1)/beta = b(j+1)/a = q + r/a with 0 <= r < a, and Gamma(q + r/a) =
# Gamma(r/a) * prod_{i<q} (r/a + i)  (the functional equation Gamma(x+1) =
# x Gamma(x)), so mu_j = (b/a) * Gamma(r/a) * prod_{i<q} (r + i a) / a^q, with
# Gamma(0/a + q) = (q-1)!.  Only Gamma(1/a) .. Gamma((a-1)/a) are transcendental.

def gamma_constants(beta, bits):
    """[None, Gamma(1/a), ..., Gamma((a-1)/a)] as exact Fractions of mpmath
    values computed at `bits` bits (beta = a/b in lowest terms)."""
    import mpmath as mpm
    beta = Fraction(beta)
    a = beta.numerator
    out = [None]
    with mpm.workprec(bits):
        for r in range(1, a):
            man, exp = mpm.gamma(mpm.mpf(r) / a).man_exp
            out.append(Fraction(int(man)) * Fraction(2) ** int(exp))
    return out


def moments_from_constants(beta, N, n, consts):
    """mu_0..mu_{2N-2} for beta = a/b from the constants of gamma_constants,
    each formed as an exact rational and truncated once to n limbs."""
    beta = Fraction(beta)
    a, b = beta.numerator, beta.denominator
    mus = []
    for j in range(2 * N - 1):
        q, r = divmod(b * (j + 1), a)
        if r == 0:
            v = Fraction(b, a) * factorial(q - 1)
        else:
            num = b
            for i in range(q):
                num *= r + i * a
            v = Fraction(num, a ** (q + 1)) * consts[r]
        mus.append(F.from_fraction(v, n))
    return mus
