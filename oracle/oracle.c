/*
 * oracle.c -- plain FP64 CPU oracle for the blocked Cholesky, pivot-free
 * LU and Gram-Schmidt QR of Camarero, "Simple, Fast and Practicable Algorithms for Cholesky, LU
 * and QR Decomposition Using Fast Rectangular Matrix Multiplication"
 * (arXiv:1812.02056).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the tests, the smoke check and the CPU-baseline leg of the
 * benchmark compare the CUDA library against.  The library never includes,
 * links or calls it, and it shares no code with the library.
 *
 * Everything is IEEE double, round-to-nearest, compiled without FMA
 * contraction (-ffp-contract=off), so each element is the exact sequence of
 * roundings written below.  Loops over independent output elements may run
 * on several OpenMP threads; no element's arithmetic depends on the thread
 * count.
 *
 * Indices are 0-based; the paper's are 1-based and inclusive (Sec. 2, the
 * paragraph after Algorithm 3).  Matrices are row-major with a leading
 * dimension: element (i, j) of X is X[i * ldx + j].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* mode bits for orc_chol / orc_lu / orc_qr */
#define ORC_FULL_SQUARE 1 /* Cholesky: update the whole trailing square, as
                             Algorithm 1 writes it (default: lower triangle,
                             the only part the column step reads). LU always
                             updates the full square.  QR: R receives all of
                             Q^T A (default: its upper triangle, zero below). */
#define ORC_SEQUENTIAL 2  /* subtract each product L_ik*L_jk from A_ij in
                             turn instead of forming S = R R^T first */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/*
 * Algorithm 1 (fast Cholesky with step s).
 *
 * A (n x n, lda) is read, lower triangle and diagonal only unless
 * ORC_FULL_SQUARE is set (then the whole square is copied and updated).
 * L (n x n, ldl) receives the factor; its strict upper triangle is zero.
 * s >= 1.  Returns 0, or c+1 when the value under the square root at column
 * c is not positive (or is NaN): the paper assumes this never happens for a
 * positive-definite input; the oracle stops there and leaves later columns
 * of L zero.
 */
int64_t orc_chol(int64_t n, int64_t s, const double *A, int64_t lda, double *L,
                 int64_t ldl, int mode) {
  if (n < 0 || s < 1) return -1;
  const int full = (mode & ORC_FULL_SQUARE) != 0;
  const int seq = (mode & ORC_SEQUENTIAL) != 0;
  /* working copy of A: the algorithm overwrites A's trailing part */
  double *W = (double *)malloc((size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1) * sizeof(double));
  if (!W) return -2;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      W[i * n + j] = (full || j <= i) ? A[i * lda + j] : 0.0;
  /* L := zero matrix of size n */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) L[i * ldl + j] = 0.0;

  int64_t z = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (c == z + s) {
      /* R := L[c..n-1, z..c-1];  S := R R^T;  A[c.., c..] -= S;  z := c */
#pragma omp parallel for schedule(dynamic, 8)
      for (int64_t i = c; i < n; ++i) {
        const int64_t jend = full ? n : i + 1;
        for (int64_t j = c; j < jend; ++j) {
          if (seq) {
            double w = W[i * n + j];
            for (int64_t k = z; k < c; ++k) w = w - L[i * ldl + k] * L[j * ldl + k];
            W[i * n + j] = w;
          } else {
            double sij = 0.0;
            for (int64_t k = z; k < c; ++k) sij = sij + L[i * ldl + k] * L[j * ldl + k];
            W[i * n + j] = W[i * n + j] - sij;
          }
        }
      }
      z = c;
    }
    /* L_cc := sqrt(A_cc - sum_{k=z}^{c-1} L_ck^2) */
    double d = W[c * n + c];
    for (int64_t k = z; k < c; ++k) d = d - L[c * ldl + k] * L[c * ldl + k];
    if (!(d > 0.0)) {
      free(W);
      return c + 1;
    }
    const double lcc = sqrt(d);
    L[c * ldl + c] = lcc;
    /* L_ic := (A_ic - sum_{k=z}^{c-1} L_ik L_ck) / L_cc   for i > c */
#pragma omp parallel for schedule(static)
    for (int64_t i = c + 1; i < n; ++i) {
      double v = W[i * n + c];
      for (int64_t k = z; k < c; ++k) v = v - L[i * ldl + k] * L[c * ldl + k];
      L[i * ldl + c] = v / lcc;
    }
  }
  free(W);
  return 0;
}

/*
 * Algorithm 2 (fast LU with step s, no pivoting): A = L U with L lower
 * triangular and U upper unitriangular.
 *
 * A (n x n, lda) is read in full.  L and U (n x n each) receive the factors;
 * the parts outside their triangles are zero.  The diagonal of U is the
 * computed quotient L_cc / L_cc, which is exactly 1 in IEEE arithmetic.
 * Returns 0, or c+1 when L_cc is zero or NaN (the paper requires nonzero
 * leading principal minors, which rules this out).
 */
int64_t orc_lu(int64_t n, int64_t s, const double *A, int64_t lda, double *L,
               int64_t ldl, double *U, int64_t ldu, int mode) {
  if (n < 0 || s < 1) return -1;
  const int seq = (mode & ORC_SEQUENTIAL) != 0;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  double *W = (double *)malloc(nn * nn * sizeof(double));
  double *urow = (double *)malloc(nn * sizeof(double)); /* row c of U being formed  */
  double *ucol = (double *)malloc(nn * sizeof(double)); /* U[z..c-1][c], gathered   */
  if (!W || !urow || !ucol) {
    free(W);
    free(urow);
    free(ucol);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) W[i * n + j] = A[i * lda + j];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      L[i * ldl + j] = 0.0;
      U[i * ldu + j] = 0.0;
    }

  /* Memory is walked by rows: a row of S (or of U) keeps one partial sum per
     element and receives the products in ascending k, so every element sees
     the same sequence of roundings as the k-innermost loop of the paper. */
  int64_t z = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (c == z + s) {
      /* R_L := L[c.., z..c-1]; R_U := U[z..c-1, c..]; S := R_L R_U;
         A[c.., c..] -= S;  z := c */
#pragma omp parallel
      {
        double *srow = (double *)malloc(nn * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = c; i < n; ++i) {
          if (seq) {
            for (int64_t k = z; k < c; ++k) {
              const double lik = L[i * ldl + k];
              for (int64_t j = c; j < n; ++j) W[i * n + j] = W[i * n + j] - lik * U[k * ldu + j];
            }
          } else {
            for (int64_t j = c; j < n; ++j) srow[j] = 0.0;
            for (int64_t k = z; k < c; ++k) {
              const double lik = L[i * ldl + k];
              for (int64_t j = c; j < n; ++j) srow[j] = srow[j] + lik * U[k * ldu + j];
            }
            for (int64_t j = c; j < n; ++j) W[i * n + j] = W[i * n + j] - srow[j];
          }
        }
        free(srow);
      }
      z = c;
    }
    /* L_ic := A_ic - sum_{k=z}^{c-1} L_ik U_kc   for i >= c */
    for (int64_t k = z; k < c; ++k) ucol[k] = U[k * ldu + c];
#pragma omp parallel for schedule(static)
    for (int64_t i = c; i < n; ++i) {
      double v = W[i * n + c];
      for (int64_t k = z; k < c; ++k) v = v - L[i * ldl + k] * ucol[k];
      L[i * ldl + c] = v;
    }
    const double lcc = L[c * ldl + c];
    if (lcc == 0.0 || lcc != lcc) {
      free(W);
      free(urow);
      free(ucol);
      return c + 1;
    }
    /* U_ci := (A_ci - sum_{k=z}^{c-1} L_ck U_ki) / L_cc   for i >= c */
#pragma omp parallel for schedule(static)
    for (int64_t i0 = c; i0 < n; i0 += 256) {
      const int64_t i1 = i0 + 256 < n ? i0 + 256 : n;
      for (int64_t i = i0; i < i1; ++i) urow[i] = W[c * n + i];
      for (int64_t k = z; k < c; ++k) {
        const double lck = L[c * ldl + k];
        for (int64_t i = i0; i < i1; ++i) urow[i] = urow[i] - lck * U[k * ldu + i];
      }
      for (int64_t i = i0; i < i1; ++i) U[c * ldu + i] = urow[i] / lcc;
    }
  }
  free(W);
  free(urow);
  free(ucol);
  return 0;
}

/*
 * Algorithm 3 (fast QR with step s): A = Q R with Q orthogonal and R upper
 * triangular.
 *
 * M starts as a copy of A.  Column c of Q is column c of M, made orthogonal
 * to the columns of Q computed since the checkpoint z one after the other
 * (v := v - u (u^T v) for u = Q[:, z], ..., Q[:, c-1]) and divided by its
 * norm.  When c = z + s, the columns c..n-1 of M first lose their
 * components along the block B_Q = Q[:, z..c-1] at once: C := B_Q^T B_M,
 * S := B_Q C, M[:, c..] -= S, z := c.  Finally R := Q^T A.
 *
 * A, Q, R are n x n (lda, ldq, ldr).  R holds (Q^T A)_ij for j >= i and zero
 * below the diagonal, or all of Q^T A with ORC_FULL_SQUARE.  Every sum runs
 * over its index in ascending order, one product at a time (the loops walk
 * rows of M and A for locality; each element still receives its products in
 * that order).  Returns 0, or c+1 when the norm of the projected column c is
 * zero or NaN (A singular): the paper assumes full rank; the oracle stops
 * there and leaves Q's later columns and R zero.
 */
int64_t orc_qr(int64_t n, int64_t s, const double *A, int64_t lda, double *Q, int64_t ldq,
               double *R, int64_t ldr, int mode) {
  if (n < 0 || s < 1) return -1;
  const int full = (mode & ORC_FULL_SQUARE) != 0;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t sw = (size_t)(s < n ? s : (n > 0 ? n : 1));
  double *M = (double *)malloc(nn * nn * sizeof(double));   /* working copy, row-major */
  double *Qc = (double *)malloc(nn * nn * sizeof(double));  /* Q by columns: Qc[j*n+i] = Q_ij */
  double *Cm = (double *)malloc(sw * nn * sizeof(double));  /* C = B_Q^T B_M, w x (n-c) */
  double *v = (double *)malloc(nn * sizeof(double));
  if (!M || !Qc || !Cm || !v) {
    free(M);
    free(Qc);
    free(Cm);
    free(v);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      M[i * n + j] = A[i * lda + j];
      Qc[j * n + i] = 0.0;
      Q[i * ldq + j] = 0.0;
      R[i * ldr + j] = 0.0;
    }

  int64_t z = 0, info = 0;
  for (int64_t c = 0; c < n && info == 0; ++c) {
    if (c == z + s) {
      const int64_t w = c - z, m = n - c;
      /* C := B_Q^T B_M:  C_kj = sum_i Q_{i,z+k} M_{i,c+j} */
#pragma omp parallel for schedule(static)
      for (int64_t k = 0; k < w; ++k) {
        double *ck = Cm + k * m;
        const double *qk = Qc + (z + k) * n;
        for (int64_t j = 0; j < m; ++j) ck[j] = 0.0;
        for (int64_t i = 0; i < n; ++i) {
          const double q = qk[i];
          const double *mi = M + i * n + c;
          for (int64_t j = 0; j < m; ++j) ck[j] = ck[j] + q * mi[j];
        }
      }
      /* S := B_Q C;  M[:, c..] -= S:  S_ij = sum_k Q_{i,z+k} C_kj */
#pragma omp parallel
      {
        double *srow = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
          for (int64_t j = 0; j < m; ++j) srow[j] = 0.0;
          for (int64_t k = 0; k < w; ++k) {
            const double q = Qc[(z + k) * n + i];
            const double *ck = Cm + k * m;
            for (int64_t j = 0; j < m; ++j) srow[j] = srow[j] + q * ck[j];
          }
          double *mi = M + i * n + c;
          for (int64_t j = 0; j < m; ++j) mi[j] = mi[j] - srow[j];
        }
        free(srow);
      }
      z = c;
    }
    /* v := column c of M;  v := v - u (u^T v) for u = Q[:, z], ..., Q[:, c-1] */
    for (int64_t i = 0; i < n; ++i) v[i] = M[i * n + c];
    for (int64_t j = z; j < c; ++j) {
      const double *u = Qc + j * n;
      double d = 0.0;
      for (int64_t i = 0; i < n; ++i) d = d + u[i] * v[i];
      for (int64_t i = 0; i < n; ++i) v[i] = v[i] - u[i] * d;
    }
    /* Q[:, c] := v / ||v|| */
    double nrm2 = 0.0;
    for (int64_t i = 0; i < n; ++i) nrm2 = nrm2 + v[i] * v[i];
    const double nrm = sqrt(nrm2);
    if (!(nrm > 0.0)) {
      info = c + 1;
      break;
    }
    for (int64_t i = 0; i < n; ++i) Qc[c * n + i] = v[i] / nrm;
  }
  if (info == 0) {
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) Q[i * ldq + j] = Qc[j * n + i];
    /* R := Q^T A:  R_ij = sum_k Q_ki A_kj */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
      const int64_t j0 = full ? 0 : i;
      double *ri = R + i * ldr;
      const double *qi = Qc + i * n;
      for (int64_t j = j0; j < n; ++j) ri[j] = 0.0;
      for (int64_t k = 0; k < n; ++k) {
        const double q = qi[k];
        const double *ak = A + k * lda;
        for (int64_t j = j0; j < n; ++j) ri[j] = ri[j] + q * ak[j];
      }
    }
  }
  free(M);
  free(Qc);
  free(Cm);
  free(v);
  return info;
}

/*
 * Triangular solves, textbook forward and back substitution, B row-major
 * n x nrhs (ldb), overwritten with the solution.
 */

/* L Y = B, L lower (non-unit diagonal) */
void orc_solve_lower(int64_t n, int64_t nrhs, const double *L, int64_t ldl, double *B,
                     int64_t ldb) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrhs; ++r) {
    for (int64_t i = 0; i < n; ++i) {
      double v = B[i * ldb + r];
      for (int64_t k = 0; k < i; ++k) v = v - L[i * ldl + k] * B[k * ldb + r];
      B[i * ldb + r] = v / L[i * ldl + i];
    }
  }
}

/* L^T X = Y, L lower (non-unit diagonal) */
void orc_solve_lower_trans(int64_t n, int64_t nrhs, const double *L, int64_t ldl, double *B,
                           int64_t ldb) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrhs; ++r) {
    for (int64_t i = n - 1; i >= 0; --i) {
      double v = B[i * ldb + r];
      for (int64_t k = i + 1; k < n; ++k) v = v - L[k * ldl + i] * B[k * ldb + r];
      B[i * ldb + r] = v / L[i * ldl + i];
    }
  }
}

/* U X = Y, U upper with unit diagonal (the stored diagonal is not read) */
void orc_solve_unit_upper(int64_t n, int64_t nrhs, const double *U, int64_t ldu, double *B,
                          int64_t ldb) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrhs; ++r) {
    for (int64_t i = n - 1; i >= 0; --i) {
      double v = B[i * ldb + r];
      for (int64_t k = i + 1; k < n; ++k) v = v - U[i * ldu + k] * B[k * ldb + r];
      B[i * ldb + r] = v;
    }
  }
}

/* X = A^{-1} B from a Cholesky factor: L Y = B, then L^T X = Y */
void orc_chol_solve(int64_t n, int64_t nrhs, const double *L, int64_t ldl, double *B,
                    int64_t ldb) {
  orc_solve_lower(n, nrhs, L, ldl, B, ldb);
  orc_solve_lower_trans(n, nrhs, L, ldl, B, ldb);
}

/* X = A^{-1} B from a Crout LU: L Y = B, then U X = Y */
void orc_lu_solve(int64_t n, int64_t nrhs, const double *L, int64_t ldl, const double *U,
                  int64_t ldu, double *B, int64_t ldb) {
  orc_solve_lower(n, nrhs, L, ldl, B, ldb);
  orc_solve_unit_upper(n, nrhs, U, ldu, B, ldb);
}

/* R = B - A X  (all row-major, n x n A, n x nrhs B, X, R) */
void orc_residual(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *X,
                  int64_t ldx, const double *B, int64_t ldb, double *R, int64_t ldr) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t r = 0; r < nrhs; ++r) {
      double v = 0.0;
      for (int64_t k = 0; k < n; ++k) v = v + A[i * lda + k] * X[k * ldx + r];
      R[i * ldr + r] = B[i * ldb + r] - v;
    }
  }
}

/*
 * Iterative refinement from a (possibly low-precision) Cholesky factor held
 * in FP64:  x := solve(L, b); repeat { r := b - A x; stop when
 * max_r eta_r <= tol; d := solve(L, r); x := x + d }.  eta_r is the normwise
 * backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) of
 * column r.  Returns the number of corrections applied; *eta_out receives
 * the final max eta (or the last one if max_iter was reached).
 */
int64_t orc_chol_refine(int64_t n, int64_t nrhs, const double *A, int64_t lda, const double *L,
                        int64_t ldl, const double *B, int64_t ldb, double *X, int64_t ldx,
                        double tol, int64_t max_iter, double *eta_out) {
  double *R = (double *)malloc((size_t)(n > 0 ? n : 1) * (size_t)(nrhs > 0 ? nrhs : 1) * sizeof(double));
  if (!R) return -2;
  double anorm = 0.0; /* ||A||_inf, max row sum of |A| */
  for (int64_t i = 0; i < n; ++i) {
    double rs = 0.0;
    for (int64_t k = 0; k < n; ++k) rs = rs + fabs(A[i * lda + k]);
    if (rs > anorm) anorm = rs;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t r = 0; r < nrhs; ++r) X[i * ldx + r] = B[i * ldb + r];
  orc_chol_solve(n, nrhs, L, ldl, X, ldx);
  int64_t it = 0;
  double eta = 0.0;
  for (;;) {
    orc_residual(n, nrhs, A, lda, X, ldx, B, ldb, R, nrhs);
    eta = 0.0;
    for (int64_t r = 0; r < nrhs; ++r) {
      double rn = 0.0, xn = 0.0, bn = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        if (fabs(R[i * nrhs + r]) > rn) rn = fabs(R[i * nrhs + r]);
        if (fabs(X[i * ldx + r]) > xn) xn = fabs(X[i * ldx + r]);
        if (fabs(B[i * ldb + r]) > bn) bn = fabs(B[i * ldb + r]);
      }
      const double den = anorm * xn + bn;
      const double e = den > 0.0 ? rn / den : 0.0;
      if (e > eta) eta = e;
    }
    if (eta <= tol || it >= max_iter) break;
    orc_chol_solve(n, nrhs, L, ldl, R, nrhs);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t r = 0; r < nrhs; ++r) X[i * ldx + r] = X[i * ldx + r] + R[i * nrhs + r];
    ++it;
  }
  if (eta_out) *eta_out = eta;
  free(R);
  return it;
}

/*
 * Backward errors, accumulated in long double:
 *   Cholesky: ||A - L L^T||_F / ||A||_F over the full square (A symmetric);
 *   LU:       ||A - L U||_F / ||A||_F.
 */
double orc_chol_backward_error(int64_t n, const double *A, int64_t lda, const double *L,
                               int64_t ldl) {
  long double num = 0.0L, den = 0.0L;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : num, den)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      long double p = 0.0L;
      const int64_t kmax = i < j ? i : j;
      for (int64_t k = 0; k <= kmax; ++k)
        p += (long double)L[i * ldl + k] * (long double)L[j * ldl + k];
      const long double a = (long double)A[i * lda + j];
      num += (a - p) * (a - p);
      den += a * a;
    }
  }
  return den > 0.0L ? (double)sqrtl(num / den) : 0.0;
}

double orc_lu_backward_error(int64_t n, const double *A, int64_t lda, const double *L,
                             int64_t ldl, const double *U, int64_t ldu) {
  long double num = 0.0L, den = 0.0L;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : num, den)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      long double p = 0.0L;
      const int64_t kmax = i < j ? i : j;
      for (int64_t k = 0; k <= kmax; ++k) {
        const long double u = (k == j) ? 1.0L : (long double)U[k * ldu + j];
        p += (long double)L[i * ldl + k] * u;
      }
      const long double a = (long double)A[i * lda + j];
      num += (a - p) * (a - p);
      den += a * a;
    }
  }
  return den > 0.0L ? (double)sqrtl(num / den) : 0.0;
}

/* ||A - Q R||_F / ||A||_F, accumulated in long double */
double orc_qr_backward_error(int64_t n, const double *A, int64_t lda, const double *Q,
                             int64_t ldq, const double *R, int64_t ldr) {
  long double num = 0.0L, den = 0.0L;
#pragma omp parallel for reduction(+ : num, den) schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      long double acc = 0.0L;
      for (int64_t k = 0; k < n; ++k)
        acc += (long double)Q[i * ldq + k] * (long double)R[k * ldr + j];
      const long double d = (long double)A[i * lda + j] - acc;
      num += d * d;
      den += (long double)A[i * lda + j] * (long double)A[i * lda + j];
    }
  return den > 0.0L ? (double)sqrtl(num / den) : 0.0;
}

/* ||Q^T Q - I||_F, accumulated in long double */
double orc_orthogonality(int64_t n, const double *Q, int64_t ldq) {
  long double num = 0.0L;
#pragma omp parallel for reduction(+ : num) schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      long double acc = 0.0L;
      for (int64_t k = 0; k < n; ++k)
        acc += (long double)Q[k * ldq + i] * (long double)Q[k * ldq + j];
      const long double d = acc - (i == j ? 1.0L : 0.0L);
      num += d * d;
    }
  return (double)sqrtl(num);
}
