"""Pins for the oracle's error measures.

The factors of Algorithms 1-3 (Sec. 2) are judged by four measures that the
oracle computes in long double:

  Cholesky   ||A - L L^T||_F / ||A||_F   (L: its lower triangle)
  Crout LU   ||A - L U||_F / ||A||_F     (U: strict upper part + unit diagonal)
  QR         ||A - Q R||_F / ||A||_F     (all entries of Q and R)
  Q          ||Q^T Q - I||_F

They are definitions, not steps of the paper.  Each is pinned here against the
same quantity computed from the definition in exact rational arithmetic
(``fractions``; the final square root in 40-digit decimal), on

  (a) integer cases whose answer is an exact rational: the Pascal factor plus
      a known integer error, random integer Q and R, a scaled Hadamard matrix
      (exactly orthogonal, measure 0) and diagonal cases with a hand value;
  (b) floating-point factors perturbed by about 1e-8 relative, far above
      rounding, so that the residual is not rounding noise;

and against numpy's norms at n = 192, where the perturbation dominates
numpy's own rounding.  A dropped square root, a missing denominator, a sum
over one triangle only, a transposed operand, an ignored unit diagonal or a
dropped identity each changes one of these values by far more than the
tolerance (tests/test_oracle_mutations.py plants them).
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests import exact

# integer cases: every sum is exact in long double, only the final division,
# square root and conversion to double round
TOL_EXACT = 1e-15
# perturbed floats: the long double sums round at 2^-64 relative to |A|,
# against a residual of about 1e-8 |A|
TOL_FLOAT = 1e-9


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _int_lower(n, seed, lo=-2, hi=2):
    return np.tril(I.rng(seed).integers(lo, hi + 1, size=(n, n))).astype(np.float64)


def _junk_upper(M, seed, k=1):
    """M with random junk in its strict upper part (from diagonal offset k)."""
    J = I.rng(seed).integers(-9, 10, size=M.shape).astype(np.float64)
    return np.tril(M, k - 1) + np.triu(J, k)


def _perturb(M, seed, eps=1e-8):
    return M * (1.0 + eps * I.rng(seed).standard_normal(M.shape))


# ---------------------------------------------------------------- Cholesky
def chol_cases():
    n = 8
    P, Lp = I.pascal_sym(n), I.pascal_lower(n)
    yield "pascal_exact_factor", P, Lp  # measure 0
    yield "pascal_plus_integer_error", P, Lp + _int_lower(n, 11)
    yield "pascal_error_junk_upper", P, _junk_upper(Lp + _int_lower(n, 12), 13)
    A = I.spd_gram(20, 21)
    yield "gram_perturbed", A, _perturb(np.linalg.cholesky(A), 22)


def lu_cases():
    n = 7
    P, Lp = I.pascal_sym(n), I.pascal_lower(n)
    U = Lp.T.copy()
    yield "pascal_exact", P, Lp, U
    L1 = Lp + _int_lower(n, 31)
    U1 = U + np.triu(I.rng(32).integers(-2, 3, size=(n, n)), 1)
    yield "pascal_plus_integer_error", P, L1, U1
    # the stored diagonal and lower part of U and the strict upper part of L
    # are not part of the factor: junk there must not change the measure
    Uj = np.triu(U1, 1) + np.tril(I.rng(33).integers(-9, 10, size=(n, n)))
    Uj[np.diag_indices(n)] = 5.0
    yield "junk_outside_factor", P, _junk_upper(L1, 34), Uj
    C = I.lu_diag_dominant(16, 35)
    Lo, Uo, _ = oracle.lu(C, 4)
    yield "crout_perturbed", C, _perturb(Lo, 36), np.triu(_perturb(Uo, 37), 1) + np.eye(16)


def qr_cases():
    n = 7
    g = I.rng(41)
    A = g.integers(-5, 6, size=(n, n)).astype(np.float64)
    Q = g.integers(-3, 4, size=(n, n)).astype(np.float64)
    R = g.integers(-3, 4, size=(n, n)).astype(np.float64)
    yield "integer_full_R", A, Q, R
    yield "integer_upper_R", A, Q, np.triu(R)
    D = I.gaussian(18, 18, 42) + 6.0 * np.eye(18)
    Qh, Rh = np.linalg.qr(D)
    yield "lapack_perturbed", D, _perturb(Qh, 43), _perturb(Rh, 44)


def orth_cases():
    H = np.array([[1.0]])
    while H.shape[0] < 4:
        H = np.block([[H, H], [H, -H]])
    yield "hadamard4_half", H / 2.0, 0.0  # exactly orthogonal
    yield "diag_2", np.diag([2.0, 1.0, 1.0]), 3.0  # Q^T Q - I = diag(3, 0, 0)
    yield "integer_unsymmetric", I.rng(51).integers(-3, 4, size=(6, 6)).astype(np.float64), None
    Qh, _ = np.linalg.qr(I.gaussian(20, 20, 52))
    yield "lapack_perturbed", _perturb(Qh, 53), None


def _tol(name):
    return TOL_FLOAT if "perturbed" in name else TOL_EXACT


def check_error_measures() -> bool:
    """Every exact case above, as one boolean (used by the mutation tests)."""
    for name, A, L in chol_cases():
        D, Af = exact.chol_residual(A, L)
        want, got = exact.frob_ratio(D, Af), oracle.chol_backward_error(A, L)
        if not (want == got == 0.0) and _rel(got, want) > _tol(name):
            return False
    for name, A, L, U in lu_cases():
        D, Af = exact.lu_residual(A, L, U)
        want, got = exact.frob_ratio(D, Af), oracle.lu_backward_error(A, L, U)
        if not (want == got == 0.0) and _rel(got, want) > _tol(name):
            return False
    for name, A, Q, R in qr_cases():
        D, Af = exact.qr_residual(A, Q, R)
        want, got = exact.frob_ratio(D, Af), oracle.qr_backward_error(A, Q, R)
        if _rel(got, want) > _tol(name):
            return False
    for name, Q, hand in orth_cases():
        want = exact.frob_ratio(exact.orthogonality_defect(Q), None)
        got = oracle.orthogonality(Q)
        if hand is not None and want != hand:
            return False
        if not (want == got == 0.0) and _rel(got, want) > _tol(name):
            return False
    return True


@pytest.mark.parametrize("case", list(chol_cases()), ids=lambda c: c[0])
def test_chol_backward_error_exact(case):
    name, A, L = case
    D, Af = exact.chol_residual(A, L)
    want = exact.frob_ratio(D, Af)
    got = oracle.chol_backward_error(A, L)
    if name == "pascal_exact_factor":
        assert want == 0.0 and got == 0.0
    else:
        assert want > 0.0
        assert _rel(got, want) <= _tol(name), (got, want)


@pytest.mark.parametrize("case", list(lu_cases()), ids=lambda c: c[0])
def test_lu_backward_error_exact(case):
    name, A, L, U = case
    D, Af = exact.lu_residual(A, L, U)
    want = exact.frob_ratio(D, Af)
    got = oracle.lu_backward_error(A, L, U)
    if name == "pascal_exact":
        assert want == 0.0 and got == 0.0
    else:
        assert want > 0.0
        assert _rel(got, want) <= _tol(name), (got, want)


@pytest.mark.parametrize("case", list(qr_cases()), ids=lambda c: c[0])
def test_qr_backward_error_exact(case):
    name, A, Q, R = case
    D, Af = exact.qr_residual(A, Q, R)
    want = exact.frob_ratio(D, Af)
    got = oracle.qr_backward_error(A, Q, R)
    assert want > 0.0
    assert _rel(got, want) <= _tol(name), (got, want)


@pytest.mark.parametrize("case", list(orth_cases()), ids=lambda c: c[0])
def test_orthogonality_exact(case):
    name, Q, hand = case
    want = exact.frob_ratio(exact.orthogonality_defect(Q), None)
    got = oracle.orthogonality(Q)
    if hand is not None:
        assert want == hand
    if want == 0.0:
        assert got == 0.0
    else:
        assert _rel(got, want) <= _tol(name), (got, want)


def test_pascal_integer_error_by_hand():
    """n = 2 by hand: A = [[1, 1], [1, 2]], L = [[1, 0], [2, 1]] gives
    L L^T = [[1, 2], [2, 5]], A - L L^T = [[0, -1], [-1, -3]]: the measure is
    sqrt(11 / 7)."""
    A = np.array([[1.0, 1.0], [1.0, 2.0]])
    L = np.array([[1.0, 0.0], [2.0, 1.0]])
    assert _rel(oracle.chol_backward_error(A, L), np.sqrt(11.0 / 7.0)) <= TOL_EXACT
    # LU of the same A with U = [[1, 3], [0, 1]]: L U = [[1, 3], [2, 7]],
    # A - L U = [[0, -2], [-1, -5]]: sqrt(30 / 7)
    U = np.array([[1.0, 3.0], [0.0, 1.0]])
    assert _rel(oracle.lu_backward_error(A, L, U), np.sqrt(30.0 / 7.0)) <= TOL_EXACT


@pytest.mark.parametrize("kind", ["chol", "lu", "qr", "orth"])
def test_against_numpy_norms_n192(kind):
    """At n = 192 with a 1e-6 perturbation numpy's FP64 residual is accurate
    to about n u / 1e-6 relative: the two must agree to 1e-6."""
    n = 192
    if kind == "chol":
        A = I.spd_gram(n, 61)
        L = np.tril(_perturb(np.linalg.cholesky(A), 62, 1e-6))
        want = np.linalg.norm(A - L @ L.T) / np.linalg.norm(A)
        got = oracle.chol_backward_error(A, L)
    elif kind == "lu":
        A = I.lu_diag_dominant(n, 63)
        Lo, Uo, _ = oracle.lu(A, 32)
        L = np.tril(_perturb(Lo, 64, 1e-6))
        U = np.triu(_perturb(Uo, 65, 1e-6), 1) + np.eye(n)
        want = np.linalg.norm(A - L @ U) / np.linalg.norm(A)
        got = oracle.lu_backward_error(A, L, U)
    elif kind == "qr":
        A = I.gaussian(n, n, 66) + 2.0 * np.sqrt(n) * np.eye(n)
        Qh, Rh = np.linalg.qr(A)
        Q, R = _perturb(Qh, 67, 1e-6), _perturb(Rh, 68, 1e-6)
        want = np.linalg.norm(A - Q @ R) / np.linalg.norm(A)
        got = oracle.qr_backward_error(A, Q, R)
    else:
        Qh, _ = np.linalg.qr(I.gaussian(n, n, 69))
        Q = _perturb(Qh, 70, 1e-6)
        want = np.linalg.norm(Q.T @ Q - np.eye(n))
        got = oracle.orthogonality(Q)
    assert want > 1e-8
    assert _rel(got, want) <= 1e-6, (got, want)


def test_zero_matrix_measures_zero():
    Z = np.zeros((4, 4))
    assert oracle.chol_backward_error(Z, Z) == 0.0
    assert oracle.lu_backward_error(Z, Z, np.eye(4)) == 0.0
    assert oracle.qr_backward_error(Z, Z, Z) == 0.0


def test_all_cases_pass():
    assert check_error_measures()
