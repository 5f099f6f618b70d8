"""Loss estimate of the truncating LDL^T and the working-precision rule.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.3 leaves the working precision to the user (the paper picks K by
trial and confirms it by doubling, Sec. 4.1).  A cheap a-posteriori measure
of what the factorisation cost: each pivot d_i is the Schur complement left
of the diagonal moment mu_{2i} = H[i][i], so log2(mu_{2i} / d_i) counts the
leading bits that cancelled in forming it.

    loss = max(0, max_i ceil(log2(mu_{2i} / d_i)))

computed here exactly from the rationals of the two numbers.  The bits the
truncating factorisation actually loses, seen by precision doubling (the
relative difference of D and lambda_1 between p and 2p bits), stay below
2 loss + 32 for beta = 1/4 ... 1 (about 1.6 to 2.3 times the estimate).  The
rule that uses it: a result is trusted to 1e-40 (133 bits) with 64 bits to
spare when
    p >= 2 loss + 32 + 133 + 64.
"""
from fractions import Fraction

from . import mpfloat as F

LOSS_FACTOR = 2
LOSS_SLACK = 32
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
    return LOSS_FACTOR * loss + LOSS_SLACK + KEEP_BITS
