"""Reading R17 (the preconditioner remark of Sec. 6): can the working
precision follow the loss still to come along the factorisation?

On the oracle (beta = 1/2, N = 96, k = 16): Algorithm 1 at a per-step width,
then Algorithm 4, the block and lambda_1 at the fixed width the precision
rule picks (2 loss + 229 bits), against lambda_1 at four times the bits.

* Fixed rule width: lambda_1 to better than 1e-70.
* Step i at 2 (loss_max - loss_i) + 229 bits (the width the remaining
  cancellation would need): 24 % less trailing-update work, but lambda_1
  is off by more than 1e-40: the late columns of L feed Algorithm 4 and the
  block at full weight, so every bit taken from them is lost at the end.
* Step i at the rule width less loss_i: 6 % less work, and still 10 or more
  digits lost.

So the variable-width variant is not built; the precision rule picks one
width per instance instead.
"""
import math
from fractions import Fraction

import pytest

mpm = pytest.importorskip("mpmath")

from oracle import eigen as EG
from oracle import invblock as IB
from oracle import ldlt as LD
from oracle import moments as M
from oracle import mpfloat as F
from oracle import precision as P


def ldlt_per_step_width(mu, N, width):
    """Algorithm 1 (Sec. 4.3) with step i's quotients and updates truncated
    to width[i] limbs (the oracle's loop, one width per step)."""
    A = [[mu[r + c] for c in range(r + 1)] for r in range(N)]
    D = [None] * N
    L = [[None] * a for a in range(N)]
    for i in range(N):
        n = width[i]
        d = A[i][i]
        D[i] = d
        B = [None] * N
        for r in range(i + 1, N):
            B[r] = F.div(A[r][i], d, n)
        for c in range(i + 1, N):
            u = A[c][i]
            for r in range(c, N):
                A[r][c] = F.fused(A[r][c], u, B[r], n)
        for r in range(i + 1, N):
            L[r][i] = B[r]
    return D, L


def lambda1(D, L, N, k, n):
    X = IB.partial_inverse(L, N, k, n)
    prec = 2 * 32 * n + 64
    with mpm.workprec(prec):
        S = IB.inverse_block(X, D, k, n)
        lam, _, _, _ = EG.lambdas(S, 1, prec)
    return lam[0]


def log10_rel(a, ref, bits):
    with mpm.workprec(bits):
        r = mpm.mpf(ref)
        d = abs(mpm.mpf(a) - r)
        return -math.inf if d == 0 else float(mpm.log10(d / r))


def test_width_cannot_follow_the_remaining_loss():
    beta, N, k = Fraction(1, 2), 96, 16
    n_hi = 4 * ((3 * N + 229) // 32 + 2)
    mu_hi = M.moments(beta, N, n_hi)
    Dh, Lh = LD.ldlt(mu_hi, N, n_hi)
    ref = lambda1(Dh, Lh, N, k, n_hi)
    loss = [max(0, P.ceil_log2(F.to_fraction(mu_hi[2 * i]) / F.to_fraction(Dh[i]))) for i in range(N)]
    lmax = max(loss)
    n_rule = -(-(2 * lmax + 229) // 32)
    mu = M.moments(beta, N, n_rule)

    def trailing_work(width):
        return sum((N - 1 - i) * (N - i) // 2 * width[i] ** 2 for i in range(N))

    fixed = [n_rule] * N
    Df, Lf = LD.ldlt(mu, N, n_rule)
    e_fixed = log10_rel(lambda1(Df, Lf, N, k, n_rule), ref, 32 * n_hi)
    assert e_fixed < -70

    remaining = [max(8, -(-(2 * (lmax - loss[i]) + 229) // 32)) for i in range(N)]
    Dv, Lv = ldlt_per_step_width(mu, N, remaining)
    e_rem = log10_rel(lambda1(Dv, Lv, N, k, n_rule), ref, 32 * n_hi)
    assert trailing_work(remaining) < 0.8 * trailing_work(fixed)
    assert e_rem > -40

    less_done = [-(-(32 * n_rule - loss[i]) // 32) for i in range(N)]
    Db, Lb = ldlt_per_step_width(mu, N, less_done)
    e_less = log10_rel(lambda1(Db, Lb, N, k, n_rule), ref, 32 * n_hi)
    assert trailing_work(less_done) > 0.9 * trailing_work(fixed)
    assert e_less > e_fixed + 10
