"""Exact rational arithmetic for brute-force pins of small factorizations.

Determinants are taken over ``fractions.Fraction`` by cofactor-free
elimination with exact pivot search; entries of the Cholesky and Crout LU
factors then follow from the classical minor formulas (D_j is the j-th
leading principal minor, D_0 = 1; rows/cols are 0-based, j is a column):

  Crout L_ij   = det A[{0..j-1, i}, {0..j}] / D_j            (i >= j)
  Crout U_ji   = det A[{0..j}, {0..j-1, i}] / D_{j+1}         (i >  j)
  Cholesky L_ij = det A[{0..j-1, i}, {0..j}] / sqrt(D_j D_{j+1})

(with the index shift D_j = det of the leading j x j block).  The square
root is taken in 50-digit decimal arithmetic.
"""
from decimal import Decimal, getcontext
from fractions import Fraction


def det(M):
    """Exact determinant of a square list-of-lists of Fractions."""
    n = len(M)
    if n == 0:
        return Fraction(1)
    a = [[Fraction(x) for x in row] for row in M]
    sign = 1
    d = Fraction(1)
    for c in range(n):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            a[c], a[p] = a[p], a[c]
            sign = -sign
        d *= a[c][c]
        for r in range(c + 1, n):
            f = a[r][c] / a[c][c]
            if f:
                for k in range(c, n):
                    a[r][k] -= f * a[c][k]
    return sign * d


def _sub(A, rows, cols):
    return [[Fraction(A[r][c]) for c in cols] for r in rows]


def leading_minors(A):
    n = len(A)
    return [det(_sub(A, range(j), range(j))) for j in range(n + 1)]


def crout_exact(A):
    """Exact Crout factors (L lower, U unit upper) as Fractions."""
    n = len(A)
    D = leading_minors(A)
    L = [[Fraction(0)] * n for _ in range(n)]
    U = [[Fraction(0)] * n for _ in range(n)]
    for j in range(n):
        for i in range(j, n):
            L[i][j] = det(_sub(A, list(range(j)) + [i], range(j + 1))) / D[j]
        U[j][j] = Fraction(1)
        for i in range(j + 1, n):
            U[j][i] = det(_sub(A, range(j + 1), list(range(j)) + [i])) / D[j + 1]
    return L, U


def cholesky_exact_decimal(A, digits=50):
    """Cholesky factor by the minor formula, as Decimals with ``digits``."""
    getcontext().prec = digits
    n = len(A)
    D = leading_minors(A)
    L = [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        den = (Decimal(D[j].numerator) / Decimal(D[j].denominator)) * \
              (Decimal(D[j + 1].numerator) / Decimal(D[j + 1].denominator))
        root = den.sqrt()
        for i in range(j, n):
            num = det(_sub(A, list(range(j)) + [i], range(j + 1)))
            L[i][j] = (Decimal(num.numerator) / Decimal(num.denominator)) / root
    return L


def _fr(M):
    """Exact binary values of a float matrix (numpy array or nested lists)."""
    return [[Fraction(float(x)) for x in row] for row in M]


def frob_ratio(D, A, digits=40):
    """``||D||_F / ||A||_F`` (``||D||_F`` when ``A`` is None) for Fraction
    matrices, with the square root of the exact rational taken in decimal."""
    getcontext().prec = digits
    num = sum(x * x for row in D for x in row)
    den = Fraction(1) if A is None else sum(x * x for row in A for x in row)
    if den == 0:
        return 0.0
    q = num / den
    return float((Decimal(q.numerator) / Decimal(q.denominator)).sqrt())


def chol_residual(A, L):
    """``A - L L^T`` exactly, with ``L`` taken as its lower triangle."""
    A, L = _fr(A), _fr(L)
    n = len(A)
    return [[A[i][j] - sum(L[i][k] * L[j][k] for k in range(min(i, j) + 1)) for j in range(n)]
            for i in range(n)], A


def lu_residual(A, L, U):
    """``A - L U`` exactly, ``L`` its lower triangle, ``U`` its strict upper
    triangle plus the unit diagonal (whatever ``U`` stores on and below it)."""
    A, L, U = _fr(A), _fr(L), _fr(U)
    n = len(A)

    def u(k, j):
        return Fraction(1) if k == j else U[k][j]

    return [[A[i][j] - sum(L[i][k] * u(k, j) for k in range(min(i, j) + 1)) for j in range(n)]
            for i in range(n)], A


def qr_residual(A, Q, R):
    """``A - Q R`` exactly, with all entries of ``Q`` and ``R`` as given."""
    A, Q, R = _fr(A), _fr(Q), _fr(R)
    n = len(A)
    return [[A[i][j] - sum(Q[i][k] * R[k][j] for k in range(n)) for j in range(n)]
            for i in range(n)], A


def orthogonality_defect(Q):
    """``Q^T Q - I`` exactly."""
    Q = _fr(Q)
    n = len(Q)
    return [[sum(Q[k][i] * Q[k][j] for k in range(n)) - (1 if i == j else 0) for j in range(n)]
            for i in range(n)]
