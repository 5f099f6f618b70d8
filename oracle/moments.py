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
