"""The whole path in the paper's order: moments -> Alg. 1 -> Alg. 4 -> block -> lambda.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
from fractions import Fraction

from . import moments as M
from . import ldlt as LD
from . import invblock as IB
from . import eigen as EG


def run(beta, N, k, n, n_eig=3, mu=None):
    """Returns a dict with mu, D, L, X, S, lambdas, trunc_errors, evals, evecs.

    beta: Fraction / (num, den); n: limbs per number (32 n bits);
    mu: optional pre-computed moments (the fuzz tests pass their own).
    """
    import mpmath as mpm
    if mu is None:
        mu = M.moments(beta, N, n)
    D, L = LD.ldlt(mu, N, n)
    k = min(k, N)
    X = IB.partial_inverse(L, N, k, n)
    prec = 2 * 32 * n + 64
    with mpm.workprec(prec):
        S = IB.inverse_block(X, D, k, n)
        lam, err, ev, vec = EG.lambdas(S, n_eig, prec)
    return dict(mu=mu, D=D, L=L, X=X, S=S, lambdas=lam, trunc_errors=err,
                evals=ev, evecs=vec, prec=prec, N=N, k=k, n=n)
