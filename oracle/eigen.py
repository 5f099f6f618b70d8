"""Eigenvalues of the k x k block of H_N^{-1} and lambda = 1/nu.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 4.2: the smallest eigenvalues of H_N are the reciprocals of the largest
eigenvalues of H_N^{-1}, and the largest eigenvalues of the top-left k x k
block approximate them.  Sec. 4.5: the paper takes the largest eigenvalues of
that block and estimates the truncation error as the difference between the
estimates from the k x k and the (k-1) x (k-1) blocks.  Here the symmetric
eigenproblem is solved by mpmath.eigsy (a library routine) at the block's
own precision.
"""


def block_eigs(S, mpm):
    """Eigenvalues of the symmetric mpmath matrix S, descending, and vectors."""
    E, Q = mpm.eigsy(S)
    k = S.rows
    order = sorted(range(k), key=lambda i: -E[i])
    evals = [E[i] for i in order]
    evecs = [[Q[r, i] for r in range(k)] for i in order]
    return evals, evecs


def lambdas(S, n_eig=3, prec=None):
    """(lambda_1..lambda_n_eig, truncation errors) from the block S.

    lambda_m = 1/nu_m with nu_1 >= nu_2 >= ... the eigenvalues of S; the
    truncation error of lambda_m is lambda_m(k) - lambda_m(k-1), using the
    leading (k-1) x (k-1) block of the same S (Sec. 4.5, Table 2).
    """
    import mpmath as mpm
    prec = prec or mpm.mp.prec
    with mpm.workprec(prec):
        k = S.rows
        ev, vec = block_eigs(S, mpm)
        lam = [1 / ev[m] for m in range(min(n_eig, k))]
        err = [None] * len(lam)
        if k >= 2:
            S1 = S[0:k - 1, 0:k - 1]
            ev1, _ = block_eigs(S1, mpm)
            for m in range(min(len(lam), k - 1)):
                err[m] = lam[m] - 1 / ev1[m]
        return lam, err, ev, vec
