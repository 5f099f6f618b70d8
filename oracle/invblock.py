"""First k columns of L^{-1} (Algorithm 4) and the k x k block of H_N^{-1}.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 4 (Sec. 4.4) runs row elimination in place on the unit-lower L,
0-based, with m = k:
    for i in 0..N-1:
      for j in i+1..N-1:
        f = A[j][i]
        if i < k:  A[j][i] = -f
        for c in 0..min(k, i)-1:  A[j][c] = A[j][c] - f * A[i][c]
After it, A[j][c] (c < k) holds X[j][c] = (L^{-1})[j][c]; the unit diagonal
X[c][c] = 1 is implicit.  Every update is one truncating fused operation in
the same format as the factorisation, applied in increasing i.

The block (Sec. 4.4 eq. "index", Sec. 4.5):
    S_ab = (H^{-1})_{ab} = sum_l X[l][a] X[l][b] / D[l]      (0 <= a, b < k)
is formed here at 2p + 64 bits with mpmath from the exact X and D (each term
and each partial sum rounded at that precision), i.e. to far better than the
working precision; it is not bit-exact with any particular summation order.
"""
from . import mpfloat as F

ONE_EXP = 0


def one(n):
    return F.from_int(1, n)


def partial_inverse(L, N, k, n):
    """Algorithm 4.  Returns X as a list of rows, X[j][c] for c < k (c <= j)."""
    k = min(k, N)
    X = [[F.ZERO] * k for _ in range(N)]
    for c in range(k):
        X[c][c] = one(n)
    for i in range(N):
        for j in range(i + 1, N):
            f = L[j][i]
            if i < k:
                X[j][i] = F.neg(f)
            for c in range(min(k, i)):
                X[j][c] = F.fused(X[j][c], f, X[i][c], n)
    return X


def inverse_block(X, D, k, n, mp=None):
    """S = (H^{-1})[0:k, 0:k] as an mpmath matrix at 2*32n + 64 bits."""
    import mpmath as mpm
    prec = 2 * 32 * n + 64
    N = len(D)
    with mpm.workprec(prec):
        Xf = [[F.to_mpf(X[l][c], mpm) for c in range(k)] for l in range(N)]
        Dinv = [1 / F.to_mpf(D[l], mpm) for l in range(N)]
        S = mpm.matrix(k, k)
        for a in range(k):
            for b in range(a, k):
                s = mpm.mpf(0)
                for l in range(max(a, b), N):
                    s += Xf[l][a] * Xf[l][b] * Dinv[l]
                S[a, b] = s
                S[b, a] = s
    return S
