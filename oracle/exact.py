"""Exact-rational references used only to pin the truncating oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``ldlt_exact``: the LDL^T of a small H_N in Fraction arithmetic, by the
  textbook column formulas  D_j = H_jj - sum_{l<j} L_jl^2 D_l,
  L_ij = (H_ij - sum_{l<j} L_il L_jl D_l) / D_j  (a different loop order
  from Algorithm 1, so an index slip in one is not repeated in the other).
* ``det_bareiss``: determinant of an integer matrix by fraction-free
  elimination, for Sylvester's criterion D_i = det H_{i+1} / det H_i.
* ``inverse_exact``: H^{-1} by Gauss-Jordan on Fractions (small N).
* beta = 1 closed forms (Laguerre weight e^{-x}, mu_j = j!):
  D_i = (i!)^2,  L_ji = C(j,i) j!/i!,  (L^{-1})_ji = (-1)^{j-i} C(j,i) j!/i!.
  These follow from H = (i+j)! = L D L^T with the Laguerre polynomials'
  coefficients; they are checked here against the Fraction factorisation
  and used to pin Algorithm 1 and Algorithm 4 at beta = 1.
"""
from fractions import Fraction
from math import comb, factorial


def ldlt_exact(H):
    N = len(H)
    D = [Fraction(0)] * N
    L = [[Fraction(0)] * N for _ in range(N)]
    for j in range(N):
        L[j][j] = Fraction(1)
        D[j] = Fraction(H[j][j]) - sum(L[j][l] ** 2 * D[l] for l in range(j))
        for i in range(j + 1, N):
            L[i][j] = (Fraction(H[i][j]) - sum(L[i][l] * L[j][l] * D[l] for l in range(j))) / D[j]
    return D, L


def det_bareiss(M):
    M = [list(map(int, row)) for row in M]
    n = len(M)
    sign, prev = 1, 1
    for k in range(n - 1):
        if M[k][k] == 0:
            for r in range(k + 1, n):
                if M[r][k] != 0:
                    M[k], M[r] = M[r], M[k]
                    sign = -sign
                    break
            else:
                return 0
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                M[i][j] = (M[i][j] * M[k][k] - M[i][k] * M[k][j]) // prev
        prev = M[k][k]
    return sign * M[n - 1][n - 1]


def inverse_exact(H):
    N = len(H)
    A = [[Fraction(H[i][j]) for j in range(N)] + [Fraction(int(i == j)) for j in range(N)]
         for i in range(N)]
    for c in range(N):
        p = next(r for r in range(c, N) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [v / piv for v in A[c]]
        for r in range(N):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [row[N:] for row in A]


def laguerre_D(i):
    return factorial(i) ** 2


def laguerre_L(j, i):
    return comb(j, i) * factorial(j) // factorial(i)


def laguerre_Linv(j, i):
    return (-1) ** (j - i) * comb(j, i) * factorial(j) // factorial(i)
