"""Loss estimate of the truncating LDL^T and the working-precision rule.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.3 leaves the working precision to the user (the paper picks K by
trial and confirms it by doubling, Sec. 4.1).  A cheap a-posteriori measure
of what the factorisation cost: each pivot d_i is the Schur complement left
of the diagonal moment mu_{2i} = H[i][i], so log2(mu_{2i} / d_i) counts the
leading bits that cancelled in forming it.

    loss = max(0, max_i ceil(log2(mu_{2i} / d_i)))

computed here exactly from the rationals of the two numbers.  The rule that
uses it: a result is trusted to 1e-40 (133 bits) with 64 bits to spare when
    p - 1.8 loss >= 133 + 64,
1.8 bounding the ratio of the loss seen by precision doubling to this
estimate (about 1.7 at beta = 1/2).
"""
from fractions import Fraction

from . import mpfloat as F

LOSS_FACTOR = Fraction(9, 5)
KEEP_BITS = 133 + 64


def ceil_log2(q):
    """The least integer t with 2^t >= q, for a rational q > 0."""
    t = q.numerator.bit_length() - q.denominator.bit_length()
    while Fraction(2) ** t < q:
        t += 1
    while Fraction(2) ** (t - 1) >= q:
        t -= 1
    return t


def loss_estimate(mu, D):
    """max(0, max_i ceil(log2(mu_{2i} / d_i))) over the positive pivots."""
    best = 0
    for i, d in enumerate(D):
        dq = F.to_fraction(d)
        if dq <= 0:
            continue
        best = max(best, ceil_log2(F.to_fraction(mu[2 * i]) / dq))
    return best


def min_bits(loss):
    """The least working precision the rule accepts for this loss."""
    v = LOSS_FACTOR * loss + KEEP_BITS
    return -((-v.numerator) // v.denominator)
