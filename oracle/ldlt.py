"""LDL^T of the Hankel matrix by the right-looking loop of Algorithm 1.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 1 (Sec. 4.3), 0-based: for each column i
    B_i[j] = A_i[j] / A_i[i]                      for j > i
    A_j[k] = A_j[k] - A_i[j] * B_i[k]             for j > i, k >= j
where A_i is column i of the lower triangle (A_i[j] is the entry in row j).
In the (row r, column c) notation used here that is
    B[r]    = trunc(A[r][i] / A[i][i])
    A[r][c] = trunc(A[r][c] - A[c][i] * B[r])      for c > i, r >= c
so the column index c supplies the unscaled pivot-column entry and the row
index r the scaled one.  No pivoting: H_N is positive definite (footnote of
Sec. 4.3); a non-positive pivot under truncation raises ``NotPositive``.

Outputs: D[i] = A[i][i] after step i, and L[r][i] = B_i[r] (unit diagonal).
"""
from . import mpfloat as F


class NotPositive(ArithmeticError):
    pass


def hankel_lower(mu, N):
    """Lower triangle of H_N = (mu_{i+j}) as a list of rows: A[r][c], c <= r."""
    return [[mu[r + c] for c in range(r + 1)] for r in range(N)]


def ldlt(mu, N, n):
    """Algorithm 1 on H_N.  Returns (D, L) with L[r][c] for c < r (lists)."""
    return ldlt_subset(mu, list(range(N)), n)


def ldlt_subset(mu, idx, n):
    """Algorithm 1 on the principal submatrix H[idx, idx] (idx increasing).

    Entry (r, c) of the factor depends only on rows/columns {0..c} U {r}
    (each update of A[r][c] at step i reads A[c][i], A[r][i], A[i][i]), so
    running the same loop on idx = [0..c] + [r] reproduces L[r][c] and
    D[0..c] of the full N x N factorisation bit for bit.  This lets a test
    sample entries of a factor whose full size is out of the oracle's reach.
    """
    m = len(idx)
    A = [[mu[idx[a] + idx[b]] for b in range(a + 1)] for a in range(m)]
    D = [None] * m
    L = [[None] * a for a in range(m)]
    for i in range(m):
        d = A[i][i]
        if d[0] <= 0:
            raise NotPositive(f"pivot {idx[i]} is not positive")
        D[i] = d
        B = [None] * m
        for r in range(i + 1, m):
            B[r] = F.div(A[r][i], d, n)
        for c in range(i + 1, m):
            u = A[c][i]
            for r in range(c, m):
                A[r][c] = F.fused(A[r][c], u, B[r], n)
        for r in range(i + 1, m):
            L[r][i] = B[r]
    return D, L


def sample_entry(mu, r, c, n):
    """L[r][c] (r > c) or D[c] (r == c) of the full factor, via ldlt_subset."""
    if r == c:
        D, _ = ldlt_subset(mu, list(range(c + 1)), n)
        return D[c]
    D, L = ldlt_subset(mu, list(range(c + 1)) + [r], n)
    return L[c + 1][c]
