"""Pins of the oracle's Algorithm 3 (fast QR, block Gram-Schmidt) to results
fixed independently of it.

* closed forms: A = P R0 (P a permutation, R0 integer upper triangular with
  a positive diagonal) gives Q = P and R = R0 exactly for every step s --
  every projection, update and norm is exact -- and A = H D (H a Sylvester
  Hadamard matrix of order 4^k, D a positive diagonal) gives Q = H / 2^k and
  R = 2^k D exactly;
* a worked 3x3 example checked by hand (tests/golden/qr3_worked.txt);
* brute force: the QR of a small integer matrix through the exact Gram
  matrix A^T A, its Cholesky factor by minors in 50-digit decimals (R), and
  Q = A R^-1 in the same precision;
* LAPACK (numpy.linalg.qr, Householder) with the signs normalised so that
  diag(R) > 0 (the QR of a nonsingular matrix is then unique);
* step agreement: s = 1 and s >= n perform the same operations (each column
  is projected against the previous ones one at a time, in the same order)
  and agree bit for bit; other steps agree to rounding;
* invariants (orthogonality, backward error, triangular R, positive
  diagonal) and the breakdown column of a rank-deficient matrix.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    mats, key = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.isalpha():
                key = line
                mats[key] = []
                continue
            mats[key].append([float(x) for x in line.split()])
    return {k: np.array(v) for k, v in mats.items()}


def perm_upper(n, seed, zero_diag_at=None):
    """A = P R0: P a seeded permutation, R0 integer upper triangular."""
    g = I.rng(seed)
    perm = g.permutation(n)
    P = np.zeros((n, n))
    P[perm, np.arange(n)] = 1.0  # column j of P is e_perm[j]
    R0 = np.triu(g.integers(-5, 6, size=(n, n)).astype(np.float64), 1)
    R0[np.diag_indices(n)] = g.integers(1, 9, size=n).astype(np.float64)
    if zero_diag_at is not None:
        R0[zero_diag_at, zero_diag_at] = 0.0
    return P @ R0, P, R0


def hadamard(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


def sign_normalised_lapack(A):
    Q, R = np.linalg.qr(A)
    d = np.sign(np.diag(R))
    return Q * d[None, :], R * d[:, None]


STEPS = [1, 2, 3, 7, 16, 40]


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
@pytest.mark.parametrize("s", STEPS)
def test_permutation_times_triangular_exact(n, s):
    A, P, R0 = perm_upper(n, 7 * n + s)
    Q, R, info = oracle.qr(A, s)
    assert info == 0
    assert np.array_equal(Q, P)
    assert np.array_equal(R, R0)


@pytest.mark.parametrize("n", [4, 16, 64])
@pytest.mark.parametrize("s", [1, 3, 8, 64])
def test_hadamard_exact(n, s):
    H = hadamard(n)
    D = np.diag(np.arange(1.0, n + 1.0))
    Q, R, info = oracle.qr(H @ D, s)
    k = int(round(np.sqrt(n)))  # n = 4^j: sqrt(n) is a power of two
    assert info == 0
    assert np.array_equal(Q, H / k)
    assert np.array_equal(R, k * D)


@pytest.mark.parametrize("s", [1, 2, 3, 5])
def test_golden_qr3(s):
    g = _read_golden("qr3_worked.txt")
    Q, R, info = oracle.qr(g["A"], s)
    assert info == 0
    assert np.abs(Q - g["W"] / 3.0).max() <= 1e-15  # a few units in the last place
    assert np.abs(R - g["R"]).max() <= 1e-14


def _qr_exact_decimal(A):
    """R from the exact Gram matrix (Cholesky by minors, 50 digits), then
    Q = A R^-1 by back substitution on the columns, in the same precision."""
    from decimal import Decimal
    n = len(A)
    G = [[sum(A[k][i] * A[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    L = exact.cholesky_exact_decimal(G)
    R = [[L[j][i] if j >= i else Decimal(0) for j in range(n)] for i in range(n)]
    Q = [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        for i in range(n):
            v = Decimal(A[i][j])
            for k in range(j):
                v -= Q[i][k] * R[k][j]
            Q[i][j] = v / R[j][j]
    return Q, R


@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (4, 3), (5, 4), (6, 5)])
def test_bruteforce_qr(n, seed):
    g = I.rng(900 + seed)
    while True:
        Ai = g.integers(-4, 5, size=(n, n))
        if abs(np.linalg.det(Ai)) > 0.5:
            break
    Qe, Re = _qr_exact_decimal(Ai.tolist())
    Qx = np.array([[float(x) for x in row] for row in Qe])
    Rx = np.array([[float(x) for x in row] for row in Re])
    # Gram-Schmidt's forward error grows with the condition number: allow
    # 10 n u cond(A) (u = 2^-53)
    tol = 10 * n * 2.0 ** -53 * np.linalg.cond(Ai.astype(np.float64))
    for s in (1, 2, n):
        Q, R, info = oracle.qr(Ai.astype(np.float64), s)
        assert info == 0
        assert np.abs(Q - Qx).max() <= tol
        assert np.abs(R - Rx).max() <= tol * np.abs(Rx).max()


@pytest.mark.parametrize("s", [1, 5, 16, 64, 100])
def test_lapack_qr(s):
    A = I.gaussian(64, 64, 11) + 8.0 * np.eye(64)  # well conditioned
    Qh, Rh = sign_normalised_lapack(A)
    Q, R, info = oracle.qr(A, s)
    assert info == 0
    assert np.abs(Q - Qh).max() <= 1e-13
    assert np.abs(R - Rh).max() <= 1e-13 * np.abs(Rh).max()


def test_step_one_and_step_n_agree_bitwise():
    A = I.gaussian(100, 100, 12)
    Q1, R1, _ = oracle.qr(A, 1)
    for s in (100, 101, 1000):
        Qs, Rs, _ = oracle.qr(A, s)
        assert np.array_equal(Q1, Qs) and np.array_equal(R1, Rs)


@pytest.mark.parametrize("s", [2, 7, 32, 99])
def test_blocked_steps_agree_to_rounding(s):
    A = I.gaussian(100, 100, 13) + 10.0 * np.eye(100)
    Q1, R1, _ = oracle.qr(A, 1)
    Qs, Rs, _ = oracle.qr(A, s)
    assert np.abs(Qs - Q1).max() <= 1e-13
    assert np.abs(Rs - R1).max() <= 1e-13 * np.abs(R1).max()


@pytest.mark.parametrize("s", [1, 16, 48])
def test_invariants_n256(s):
    n = 256
    A = I.gaussian(n, n, 14) + 16.0 * np.eye(n)
    Q, R, info = oracle.qr(A, s)
    assert info == 0
    assert oracle.orthogonality(Q) <= 1e-14 * n
    assert oracle.qr_backward_error(A, Q, R) <= 1e-15 * n
    assert np.all(np.diag(R) > 0)
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n)))
    _, Rf, _ = oracle.qr(A, s, full_r=True)
    assert np.array_equal(np.triu(Rf), R)  # same sums on and above the diagonal
    assert np.abs(np.tril(Rf, -1)).max() <= 1e-14 * np.abs(A).max() * np.sqrt(n)


@pytest.mark.parametrize("c", [0, 5, 19])
@pytest.mark.parametrize("s", [1, 4, 20])
def test_breakdown_reports_column(c, s):
    """A = P R0 with R0_cc = 0: the projected column c is exactly zero."""
    A, _, _ = perm_upper(20, 40 + c, zero_diag_at=c)
    Q, R, info = oracle.qr(A, s)
    assert info == c + 1


def test_zero_order_and_bad_step():
    Q, R, info = oracle.qr(np.zeros((0, 0)), 4)
    assert info == 0 and Q.shape == (0, 0)
    with pytest.raises(ValueError):
        oracle.qr(np.eye(3), 0)
