"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a transposed
operand, a wrong index or range, a missing step) in a copy of oracle.c,
compiles the copy with the same flags, and checks that at least one pin --
Pascal closed form, rational brute force, LAPACK, step agreement, the error
measures against their exact values -- fails
with it.  The planted copies live in a temporary directory; the committed
oracle is untouched.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests import exact, test_oracle_error_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTATIONS = {
    "chol_diag_dropped_term": ("d = d - L[c * ldl + k] * L[c * ldl + k];", "d = d;"),
    "chol_diag_sign": ("d = d - L[c * ldl + k] * L[c * ldl + k];",
                       "d = d + L[c * ldl + k] * L[c * ldl + k];"),
    "chol_col_sign": ("v = v - L[i * ldl + k] * L[c * ldl + k];",
                      "v = v + L[i * ldl + k] * L[c * ldl + k];"),
    "chol_col_transposed": ("v = v - L[i * ldl + k] * L[c * ldl + k];",
                            "v = v - L[k * ldl + i] * L[c * ldl + k];"),
    "chol_no_divide": ("L[i * ldl + c] = v / lcc;", "L[i * ldl + c] = v;"),
    "chol_no_sqrt": ("const double lcc = sqrt(d);", "const double lcc = d;"),
    "chol_update_transposed": ("sij = sij + L[i * ldl + k] * L[j * ldl + k];",
                               "sij = sij + L[i * ldl + k] * L[k * ldl + j];"),
    "chol_update_sign": ("W[i * n + j] = W[i * n + j] - sij;", "W[i * n + j] = W[i * n + j] + sij;"),
    "chol_update_skips_diag": ("for (int64_t j = c; j < jend; ++j) {", "for (int64_t j = c + 1; j < jend; ++j) {"),
    "chol_checkpoint_not_moved": ("      z = c;\n    }\n    /* L_cc", "    }\n    /* L_cc"),
    "chol_col_first_term_dropped": ("for (int64_t k = z; k < c; ++k) v = v - L[i * ldl + k] * L[c * ldl + k];",
                                    "for (int64_t k = z + 1; k < c; ++k) v = v - L[i * ldl + k] * L[c * ldl + k];"),
    "lu_no_divide": ("U[c * ldu + i] = urow[i] / lcc;", "U[c * ldu + i] = urow[i];"),
    "lu_update_transposed": ("srow[j] = srow[j] + lik * U[k * ldu + j];",
                             "srow[j] = srow[j] + lik * U[j * ldu + k];"),
    "lu_col_wrong_factor": ("ucol[k] = U[k * ldu + c];", "ucol[k] = U[c * ldu + k];"),
    "lu_row_sign": ("urow[i] = urow[i] - lck * U[k * ldu + i];",
                    "urow[i] = urow[i] + lck * U[k * ldu + i];"),
    "qr_proj_sign": ("v[i] = v[i] - u[i] * d;", "v[i] = v[i] + u[i] * d;"),
    "qr_proj_dropped": ("for (int64_t i = 0; i < n; ++i) v[i] = v[i] - u[i] * d;",
                        "(void)d;"),
    "qr_first_proj_skipped": ("for (int64_t j = z; j < c; ++j) {\n      const double *u",
                              "for (int64_t j = z + 1; j < c; ++j) {\n      const double *u"),
    "qr_no_normalise": ("Qc[c * n + i] = v[i] / nrm;", "Qc[c * n + i] = v[i];"),
    "qr_update_sign": ("mi[j] = mi[j] - srow[j];", "mi[j] = mi[j] + srow[j];"),
    "qr_update_c_transposed": ("const double *qk = Qc + (z + k) * n;",
                               "const double *qk = Qc + (z + k);"),
    "qr_update_skipped_column": ("const double *mi = M + i * n + c;",
                                 "const double *mi = M + i * n + c + 1;"),
    "qr_checkpoint_not_moved": ("      z = c;\n    }\n    /* v := column c",
                                "    }\n    /* v := column c"),
    "qr_r_transposed": ("const double *qi = Qc + i * n;", "const double *qi = Qc + i;"),
    "lu_update_first_term_dropped": ("for (int64_t k = z; k < c; ++k) {\n              const double lik = L[i * ldl + k];\n              for (int64_t j = c; j < n; ++j) srow[j]",
                                     "for (int64_t k = z + 1; k < c; ++k) {\n              const double lik = L[i * ldl + k];\n              for (int64_t j = c; j < n; ++j) srow[j]"),
    # error measures (the definitions that judge every factor)
    "be_chol_no_sqrt": ("sqrtl(num / den) : 0.0;\n}\n\ndouble orc_lu_backward_error",
                        "(num / den) : 0.0;\n}\n\ndouble orc_lu_backward_error"),
    "be_chol_no_den": ("sqrtl(num / den) : 0.0;\n}\n\ndouble orc_lu_backward_error",
                       "sqrtl(num) : 0.0;\n}\n\ndouble orc_lu_backward_error"),
    "be_chol_lower_triangle_only": (
        "for (int64_t j = 0; j < n; ++j) {\n      long double p = 0.0L;\n      const int64_t kmax = i < j ? i : j;\n      for (int64_t k = 0; k <= kmax; ++k)\n        p +=",
        "for (int64_t j = 0; j <= i; ++j) {\n      long double p = 0.0L;\n      const int64_t kmax = i < j ? i : j;\n      for (int64_t k = 0; k <= kmax; ++k)\n        p +="),
    "be_chol_diag_term_dropped": (
        "for (int64_t k = 0; k <= kmax; ++k)\n        p += (long double)L[i * ldl + k] * (long double)L[j * ldl + k];",
        "for (int64_t k = 0; k < kmax; ++k)\n        p += (long double)L[i * ldl + k] * (long double)L[j * ldl + k];"),
    "be_chol_reads_upper": (
        "for (int64_t k = 0; k <= kmax; ++k)\n        p += (long double)L[i * ldl + k] * (long double)L[j * ldl + k];",
        "for (int64_t k = 0; k < n; ++k)\n        p += (long double)L[i * ldl + k] * (long double)L[j * ldl + k];"),
    "be_lu_stored_diag_used": ("const long double u = (k == j) ? 1.0L : (long double)U[k * ldu + j];",
                               "const long double u = (long double)U[k * ldu + j];"),
    "be_lu_transposed": ("p += (long double)L[i * ldl + k] * u;", "p += (long double)L[k * ldl + i] * u;"),
    "be_lu_no_sqrt": ("sqrtl(num / den) : 0.0;\n}\n\n/* ||A - Q R||_F",
                      "(num / den) : 0.0;\n}\n\n/* ||A - Q R||_F"),
    "be_lu_no_den": ("sqrtl(num / den) : 0.0;\n}\n\n/* ||A - Q R||_F",
                     "sqrtl(num) : 0.0;\n}\n\n/* ||A - Q R||_F"),
    "be_qr_no_sqrt": ("sqrtl(num / den) : 0.0;\n}\n\n/* ||Q^T Q - I||_F",
                      "(num / den) : 0.0;\n}\n\n/* ||Q^T Q - I||_F"),
    "be_qr_no_den": ("sqrtl(num / den) : 0.0;\n}\n\n/* ||Q^T Q - I||_F",
                     "sqrtl(num) : 0.0;\n}\n\n/* ||Q^T Q - I||_F"),
    "be_qr_transposed": ("acc += (long double)Q[i * ldq + k] * (long double)R[k * ldr + j];",
                         "acc += (long double)Q[k * ldq + i] * (long double)R[k * ldr + j];"),
    "be_qr_upper_r_only": ("acc += (long double)Q[i * ldq + k] * (long double)R[k * ldr + j];",
                           "if (k <= j) acc += (long double)Q[i * ldq + k] * (long double)R[k * ldr + j];"),
    "orth_no_sqrt": ("return (double)sqrtl(num);", "return (double)num;"),
    "orth_no_identity": ("const long double d = acc - (i == j ? 1.0L : 0.0L);",
                         "const long double d = acc;"),
    "orth_transposed_operand": ("acc += (long double)Q[k * ldq + i] * (long double)Q[k * ldq + j];",
                                "acc += (long double)Q[k * ldq + i] * (long double)Q[j * ldq + k];"),
    "orth_upper_only": ("const long double d = acc - (i == j ? 1.0L : 0.0L);\n      num += d * d;",
                        "const long double d = acc - (i == j ? 1.0L : 0.0L);\n      if (j >= i) num += d * d;"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation {name} does not apply"
    mutated = src.replace(old, new)
    c_path = tmp_path / f"{name}.c"
    so_path = tmp_path / f"{name}.so"
    c_path.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    str(c_path), "-o", str(so_path), "-lm"], check=True)
    return str(so_path)


def _pins_pass() -> bool:
    """Run a compact set of the pins against whatever library oracle._lib is."""
    try:
        P, Lp = I.pascal_sym(12), I.pascal_lower(12)
        for s in (1, 3, 12):
            L, info = oracle.chol(P, s)
            if info != 0 or not np.array_equal(L, Lp):
                return False
            Lu, Uu, info = oracle.lu(P, s)
            if info != 0 or not np.array_equal(Lu, Lp) or not np.array_equal(Uu, Lp.T):
                return False
        A = I.small_int_spd(5, 501)
        ref = exact.cholesky_exact_decimal(A.astype(int).tolist())
        for s in (1, 2, 5):
            L, info = oracle.chol(A, s)
            if info != 0:
                return False
            for i in range(5):
                for j in range(i + 1):
                    if abs(L[i, j] - float(ref[i][j])) > 1e-13 * max(abs(float(ref[i][j])), 1.0):
                        return False
        B = I.spd_gram(64, 3)
        ref = np.linalg.cholesky(B)
        for s in (1, 5, 64):
            L, info = oracle.chol(B, s)
            if info != 0 or np.abs(L - ref).max() > 1e-12 * np.abs(ref).max():
                return False
        C = I.lu_diag_dominant(30, 2)
        for s in (1, 4, 30):
            L, U, info = oracle.lu(C, s)
            if info != 0 or oracle.lu_backward_error(C, L, U) > 1e-13:
                return False
        # Algorithm 3: permutation times triangular (exact) and LAPACK
        g = I.rng(77)
        n = 12
        perm = g.permutation(n)
        P = np.zeros((n, n))
        P[perm, np.arange(n)] = 1.0
        R0 = np.triu(g.integers(-5, 6, size=(n, n)).astype(np.float64), 1)
        R0[np.diag_indices(n)] = g.integers(1, 9, size=n).astype(np.float64)
        for s in (1, 3, 12):
            Q, R, info = oracle.qr(P @ R0, s)
            if info != 0 or not np.array_equal(Q, P) or not np.array_equal(R, R0):
                return False
        D = I.gaussian(40, 40, 5) + 6.0 * np.eye(40)
        Qh, Rh = np.linalg.qr(D)
        sg = np.sign(np.diag(Rh))
        Qh, Rh = Qh * sg[None, :], Rh * sg[:, None]
        for s in (1, 4, 40):
            Q, R, info = oracle.qr(D, s)
            if info != 0 or np.abs(Q - Qh).max() > 1e-12 or np.abs(R - Rh).max() > 1e-11:
                return False
        # s = 1 and s = n perform the same operations in the same order
        Q1, R1, _ = oracle.qr(D, 1)
        Qn, Rn, _ = oracle.qr(D, 40)
        if not (np.array_equal(Q1, Qn) and np.array_equal(R1, Rn)):
            return False
        # the error measures against their exact values
        return test_oracle_error_pins.check_error_measures()
    except Exception:
        return False


def test_unmutated_oracle_passes_compact_pins():
    assert _pins_pass()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    path = _build_mutant(tmp_path, name, old, new)
    saved = oracle._lib
    try:
        lib = ctypes.CDLL(path)
        oracle._lib = None
        real = oracle.build
        oracle.build = lambda force=False: path  # load the planted copy
        try:
            oracle._load()
        finally:
            oracle.build = real
        assert not _pins_pass(), f"planted mistake {name} went unnoticed"
    finally:
        oracle._lib = saved
        del lib
