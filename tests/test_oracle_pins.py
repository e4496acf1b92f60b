"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

* closed form: symmetric Pascal = lower Pascal x its transpose (bit-exact);
* hand-checked worked examples under tests/golden/;
* exact recovery of integer factors;
* brute force over the rationals at n <= 8 (minor formulas);
* the paper's own special cases (Sec. 2, after Algorithm 3): s = 1 is the
  recursive (right-looking) algorithm and s = n is Cholesky-Crout, so with
  sequential subtraction every s gives the same bits;
* invariants (lower triangular, positive diagonal, backward error);
* LAPACK (numpy / torch) on the same matrices.
"""
import os
from decimal import Decimal

import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    mats, cur, key = {}, None, None
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


STEPS = [1, 2, 3, 5, 7, 16, 33]


# ---------------------------------------------------------------- closed form
@pytest.mark.parametrize("n", [1, 2, 5, 16, 26])
@pytest.mark.parametrize("s", [1, 2, 3, 7, 16, 40])
@pytest.mark.parametrize("mode", ["literal", "full", "sequential"])
def test_pascal_cholesky_exact(n, s, mode):
    P, Lp = I.pascal_sym(n), I.pascal_lower(n)
    L, info = oracle.chol(P, s, full_square=(mode == "full"), sequential=(mode == "sequential"))
    assert info == 0
    assert np.array_equal(L, Lp)


@pytest.mark.parametrize("n", [1, 3, 16, 26])
@pytest.mark.parametrize("s", [1, 2, 5, 16, 30])
def test_pascal_lu_exact(n, s):
    P, Lp = I.pascal_sym(n), I.pascal_lower(n)
    L, U, info = oracle.lu(P, s)
    assert info == 0
    assert np.array_equal(L, Lp)
    assert np.array_equal(U, Lp.T)


@pytest.mark.parametrize("s", STEPS)
def test_golden_chol3(s):
    g = _read_golden("chol3_textbook.txt")
    L, info = oracle.chol(g["A"], s)
    assert info == 0 and np.array_equal(L, g["L"])


@pytest.mark.parametrize("s", STEPS)
def test_golden_lu3(s):
    g = _read_golden("lu3_textbook.txt")
    L, U, info = oracle.lu(g["A"], s)
    assert info == 0 and np.array_equal(L, g["L"]) and np.array_equal(U, g["U"])


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("s", [1, 4, 9, 40])
def test_integer_factor_recovered_exactly(seed, s):
    n = 40
    L0 = I.unit_lower_integer(n, seed)
    A = L0 @ L0.T  # small integers: exact in FP64
    L, info = oracle.chol(A, s)
    assert info == 0 and np.array_equal(L, L0)
    U0 = I.unit_lower_integer(n, seed + 100).T
    B = L0 @ U0
    Lb, Ub, info = oracle.lu(B, s)
    assert info == 0 and np.array_equal(Lb, L0) and np.array_equal(Ub, U0)


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("seed", range(3))
def test_bruteforce_cholesky(n, seed):
    A = I.small_int_spd(n, 500 + seed)
    ref = exact.cholesky_exact_decimal(A.astype(int).tolist())
    for s in (1, 2, 3, n):
        L, info = oracle.chol(A, s)
        assert info == 0
        for i in range(n):
            for j in range(n):
                if j > i:
                    assert L[i, j] == 0.0
                    continue
                r = ref[i][j]
                err = abs(Decimal(L[i, j]) - r)
                assert err <= Decimal("1e-14") * max(abs(r), Decimal(1)), (i, j, s)


@pytest.mark.parametrize("n", [1, 2, 4, 8])
@pytest.mark.parametrize("seed", range(3))
def test_bruteforce_crout_lu(n, seed):
    rng = I.rng(700 + seed)
    A = rng.integers(-4, 5, size=(n, n)).astype(np.float64) + 9.0 * np.eye(n)
    Lx, Ux = exact.crout_exact(A.astype(int).tolist())
    for s in (1, 3, n):
        L, U, info = oracle.lu(A, s)
        assert info == 0
        for i in range(n):
            for j in range(n):
                lr, ur = float(Lx[i][j]), float(Ux[i][j])
                assert abs(L[i, j] - lr) <= 1e-14 * max(abs(lr), 1.0)
                assert abs(U[i, j] - ur) <= 1e-14 * max(abs(ur), 1.0)


# ------------------------------------------------------ the paper's special cases
def test_step_agreement_sequential_bitwise():
    """Sequential subtraction applies every product in ascending k for all s,
    so the factor is the same bits for every step (Sec. 2: s = 1 recursive,
    s = n Crout, and the correctness argument that reduces to both)."""
    n = 150
    A = I.spd_gram(n, I.seed_for(I.W_SMALL, 7))
    L1, _ = oracle.chol(A, 1, sequential=True)
    for s in [2, 3, 7, 32, 117, n - 1, n, n + 5]:
        Ls, info = oracle.chol(A, s, sequential=True)
        assert info == 0 and np.array_equal(Ls, L1), s
    # literal S-first subtraction at s = 1 and s >= n is the same sequence
    La, _ = oracle.chol(A, 1)
    Lb, _ = oracle.chol(A, n)
    Lc, _ = oracle.chol(A, n + 5)
    assert np.array_equal(La, L1) and np.array_equal(Lb, L1) and np.array_equal(Lc, L1)
    # LU likewise
    B = I.lu_diag_dominant(n, 11)
    M1 = oracle.lu(B, 1, sequential=True)
    for s in [2, 7, 64, n, n + 3]:
        Ms = oracle.lu(B, s, sequential=True)
        assert np.array_equal(Ms[0], M1[0]) and np.array_equal(Ms[1], M1[1]), s
    assert np.array_equal(oracle.lu(B, 1)[0], oracle.lu(B, n)[0])


def test_full_square_matches_lower_only_bitwise():
    """The column step reads only the lower triangle, so updating the whole
    square (as Algorithm 1 is written) cannot change L."""
    A = I.spd_gram(97, 5)
    for s in [1, 4, 10, 97]:
        assert np.array_equal(oracle.chol(A, s)[0], oracle.chol(A, s, full_square=True)[0])


def test_step_agreement_n512_tolerance():
    A = I.spd_gram(512, I.seed_for(I.W_SMALL))
    L1, _ = oracle.chol(A, 1)
    mx = np.abs(L1).max()
    for s in [2, 3, 7, 32, 117, 511, 512, 517]:
        Ls, info = oracle.chol(A, s)
        assert info == 0
        assert np.abs(Ls - L1).max() <= 1e-13 * mx, s


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("s", [1, 32, 117, 512])
def test_invariants_n512(s):
    n = 512
    A = I.spd_gram(n, I.seed_for(I.W_SMALL))
    L, info = oracle.chol(A, s)
    assert info == 0
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.all(np.diag(L) > 0)
    assert oracle.chol_backward_error(A, L) <= 1e-14 * n


def test_lu_invariants():
    n = 200
    A = I.lu_diag_dominant(n, 3)
    L, U, info = oracle.lu(A, 32)
    assert info == 0
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.all(np.tril(U, -1) == 0.0)
    assert np.all(np.diag(U) == 1.0)
    assert oracle.lu_backward_error(A, L, U) <= 1e-14 * n


# ---------------------------------------------------------------- breakdown
def test_breakdown_reports_column():
    assert oracle.chol(np.array([[-1.0]]), 1)[1] == 1
    assert oracle.chol(np.array([[1.0, 2.0], [2.0, 1.0]]), 1)[1] == 2
    A = I.spd_gram(40, 1)
    A[17, 17] = -1e6
    for s in [1, 5, 40]:
        assert oracle.chol(A, s)[1] == 18
    B = np.array([[1.0, 1.0], [1.0, 1.0]])
    assert oracle.lu(B, 1)[2] == 2
    Bn = I.lu_diag_dominant(10, 1)
    Bn[0, 0] = np.nan
    assert oracle.lu(Bn, 3)[2] == 1


# ------------------------------------------------------------ library checks
def test_numpy_cholesky_n512():
    A = I.spd_gram(512, I.seed_for(I.W_SMALL))
    L, _ = oracle.chol(A, 32)
    ref = np.linalg.cholesky(A)
    assert np.abs(L - ref).max() <= 1e-13 * np.abs(ref).max()


def test_lapack_lu_without_interchanges():
    """Partial pivoting makes no interchange on a column diagonally dominant
    matrix, so LAPACK's Doolittle factors rescale to the Crout ones."""
    import scipy.linalg
    n = 300
    A = I.lu_diag_dominant(n, 9)
    P, Ld, Ud = scipy.linalg.lu(A)
    assert np.array_equal(P, np.eye(n))
    d = np.diag(Ud)
    Lc, Uc = Ld * d[None, :], Ud / d[:, None]
    L, U, info = oracle.lu(A, 40)
    assert info == 0
    assert np.abs(L - Lc).max() <= 1e-13 * np.abs(Lc).max()
    assert np.abs(U - Uc).max() <= 1e-13 * max(np.abs(Uc).max(), 1.0)


# ------------------------------------------------------------------ solves
def test_solves_against_numpy():
    n, r = 120, 5
    A = I.spd_gram(n, 2)
    B = I.rhs(n, r, 3)
    L, _ = oracle.chol(A, 16)
    X = oracle.chol_solve(L, B)
    assert np.abs(X - np.linalg.solve(A, B)).max() <= 1e-12 * np.abs(X).max()
    C = I.lu_diag_dominant(n, 4)
    Lc, Uc, _ = oracle.lu(C, 16)
    Y = oracle.lu_solve(Lc, Uc, B)
    assert np.abs(Y - np.linalg.solve(C, B)).max() <= 1e-12 * np.abs(Y).max()
    R = oracle.residual(A, X, B)
    assert np.abs(R - (B - A @ X)).max() <= 1e-12 * np.abs(B).max()


def test_refinement_from_perturbed_factor():
    """A factor rounded to FP32 still refines to FP64 backward error."""
    n, r = 200, 4
    A = I.spd_logspaced(n, 8, cond=1e4)
    B = I.rhs(n, r, 9)
    L, _ = oracle.chol(A, 32)
    Lf = L.astype(np.float32).astype(np.float64)
    X, it, eta = oracle.chol_refine(A, Lf, B, tol=1e-15, max_iter=20)
    assert eta <= 1e-15 and 1 <= it <= 10
    assert np.abs(X - np.linalg.solve(A, B)).max() <= 1e-10 * np.abs(X).max()
