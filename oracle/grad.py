"""d lambda_1 / d beta for the k x k block estimate lambda_1 = 1/nu_1.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper computes lambda_1 only.  Its derivative follows from first-order
perturbation of the largest eigenvalue nu_1 of S = E_k^T H^{-1} E_k
(Sec. 4.2, Sec. 4.4 eq. "index"):
    d nu_1 = u^T dS u,   dS = -E_k^T H^{-1} dH H^{-1} E_k,   |u| = 1
so with w = H^{-1} E_k u = L^{-T} D^{-1} X u  (X = first k columns of L^{-1})
    d lambda_1 / d beta = (w^T Hdot w) / nu_1^2,
    w^T Hdot w = sum_s mudot_s c_s,  c_s = sum_{i+j=s} w_i w_j,
    mudot_s = d mu_s / d beta = -(mu_s / beta) (1 + x psi(x)),  x = (s+1)/beta
with psi the digamma function (derivative of eq. "moments").

``analytic_grad`` evaluates that formula at 2p + 64 bits from the oracle's own
L, D, X and the block eigenvector.  ``fd_grad`` is an independent check: a
central difference of the whole oracle pipeline at beta +- h with moments
from mpmath's Gamma.
"""
from fractions import Fraction

from . import mpfloat as F
from . import moments as M
from . import ldlt as LD
from . import invblock as IB
from . import eigen as EG


def psi_gauss(r, m, mpm):
    """psi(r/m) for 0 < r < m by Gauss's digamma theorem:
    -gamma - ln(2m) - (pi/2) cot(pi r/m)
           + 2 sum_{j=1}^{floor((m-1)/2)} cos(2 pi j r/m) ln sin(pi j/m)
    (elementary functions only, so cheap at thousands of bits)."""
    v = -mpm.euler - mpm.log(2 * m) - mpm.pi / 2 * mpm.cot(mpm.pi * r / m)
    for j in range(1, (m - 1) // 2 + 1):
        v += 2 * mpm.cos(2 * mpm.pi * j * r / m) * mpm.log(mpm.sin(mpm.pi * j / m))
    return v


def psi(x, mpm):
    """Digamma at x > 0.  A positive integer x: the exact identity
    psi(x) = H_{x-1} - gamma (harmonic number as an exact Fraction, Euler's
    gamma from mpmath).  A non-integer Fraction x = q + r/m: the recurrence
    psi(y + 1) = psi(y) + 1/y (from Gamma(y + 1) = y Gamma(y)) down to r/m,
    the q reciprocals summed exactly, plus Gauss's theorem at r/m.
    Anything else: mpmath.digamma."""
    if isinstance(x, int) or (isinstance(x, Fraction) and x.denominator == 1):
        x = int(x)
        h = Fraction(0)
        for j in range(1, x):
            h += Fraction(1, j)
        return mpm.mpf(h.numerator) / h.denominator - mpm.euler
    if isinstance(x, Fraction) and x > 0:
        m = x.denominator
        q, r = divmod(x.numerator, m)
        h = Fraction(0)
        for i in range(q):
            h += Fraction(m, r + i * m)
        return psi_gauss(r, m, mpm) + mpm.mpf(h.numerator) / h.denominator
    return mpm.digamma(x)


def analytic_grad(beta, mu_exact, L, D, X, k, n):
    """d lambda_1/d beta from the factor (L, D, X) of H at beta.

    mu_exact(s) must return mu_s as an mpmath number (exact or at >= 2p bits).
    Returns (dlambda, lambda_1, nu_1).
    """
    import mpmath as mpm
    N = len(D)
    prec = 2 * 32 * n + 64
    with mpm.workprec(prec):
        S = IB.inverse_block(X, D, k, n)
        ev, vec = EG.block_eigs(S, mpm)
        nu = ev[0]
        u = vec[0]
        norm = mpm.sqrt(sum(x * x for x in u))
        u = [x / norm for x in u]
        # z = X u, y = D^{-1} z
        y = [sum(F.to_mpf(X[l][c], mpm) * u[c] for c in range(min(k, l + 1)))
             / F.to_mpf(D[l], mpm) for l in range(N)]
        # back substitution L^T w = y
        w = [None] * N
        for i in range(N - 1, -1, -1):
            s = y[i]
            for j in range(i + 1, N):
                s -= F.to_mpf(L[j][i], mpm) * w[j]
            w[i] = s
        b = mpm.mpf(beta.numerator) / beta.denominator if isinstance(beta, Fraction) else mpm.mpf(beta)
        total = mpm.mpf(0)
        for s_ in range(2 * N - 1):
            c = mpm.mpf(0)
            for i in range(max(0, s_ - N + 1), min(s_, N - 1) + 1):
                c += w[i] * w[s_ - i]
            xq = Fraction(s_ + 1) / Fraction(beta)   # (s+1)/beta, exact
            x = mpm.mpf(xq.numerator) / xq.denominator
            mudot = -(mu_exact(s_) / b) * (1 + x * psi(xq, mpm))
            total += mudot * c
        return total / (nu * nu), 1 / nu, nu


def lambda1_at(beta_mp, N, k, n):
    """lambda_1 of the k x k block for a (possibly irrational) beta."""
    import mpmath as mpm
    mu = M.gamma_moments(beta_mp, N, n)
    D, L = LD.ldlt(mu, N, n)
    X = IB.partial_inverse(L, N, k, n)
    with mpm.workprec(2 * 32 * n + 64):
        S = IB.inverse_block(X, D, k, n)
        ev, _ = EG.block_eigs(S, mpm)
        return 1 / ev[0]


def fd_grad(beta, N, k, n, h_exp=-30):
    """Central difference (lambda(beta+h) - lambda(beta-h)) / 2h, h = 10^h_exp."""
    import mpmath as mpm
    with mpm.workprec(32 * n + 128):
        b = mpm.mpf(beta.numerator) / beta.denominator
        h = mpm.mpf(10) ** h_exp
        lp = lambda1_at(b + h, N, k, n)
        lm = lambda1_at(b - h, N, k, n)
    with mpm.workprec(2 * 32 * n + 64):
        return (lp - lm) / (2 * h)
