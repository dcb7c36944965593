"""Exact-arithmetic references used to pin the oracle (tests only).

* ``leibniz_det``: determinant from the permutation expansion (brute force).
* ``rational_gepp``: Gaussian elimination with partial pivoting in exact
  rational arithmetic (fractions.Fraction), first-index tie-break.  It gives
  the exact pivot sequence and exact L, U for small integer matrices.
"""
from fractions import Fraction
from itertools import permutations


def perm_sign(p):
    p = list(p)
    s = 1
    for i in range(len(p)):
        while p[i] != i:
            j = p[i]
            p[i], p[j] = p[j], p[i]
            s = -s
    return s


def leibniz_det(A):
    n = len(A)
    total = Fraction(0)
    for p in permutations(range(n)):
        term = Fraction(perm_sign(p))
        for i in range(n):
            term *= Fraction(A[i][p[i]])
        total += term
    return total


def rational_gepp(A, forced=None):
    """Return (ipiv 1-based, L, U) as lists of Fractions; raises on singular.

    ``forced``: optional 1-based pivot rows imposed at some steps (0 = search)."""
    n = len(A)
    M = [[Fraction(x) for x in row] for row in A]
    ipiv = []
    for j in range(n):
        p = j
        for i in range(j + 1, n):
            if abs(M[i][j]) > abs(M[p][j]):
                p = i
        if forced is not None and forced[j] > 0:
            p = forced[j] - 1
        ipiv.append(p + 1)
        if M[p][j] == 0:
            raise ZeroDivisionError("singular")
        M[j], M[p] = M[p], M[j]
        for i in range(j + 1, n):
            M[i][j] = M[i][j] / M[j][j]
            for c in range(j + 1, n):
                M[i][c] -= M[i][j] * M[j][c]
    L = [[(M[i][c] if c < i else Fraction(int(c == i))) for c in range(n)] for i in range(n)]
    U = [[(M[i][c] if c >= i else Fraction(0)) for c in range(n)] for i in range(n)]
    return ipiv, L, U
