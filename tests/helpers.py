"""Shared helpers of the test suite (comparison metrics, device handles)."""
import numpy as np


def guarded_rel_err(got, ref, floor: float = 1e-6) -> float:
    """max |got - ref| / max(|ref|, floor * max|ref|), elementwise."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    scale = np.maximum(np.abs(ref), floor * max(np.abs(ref).max(), 1e-300))
    return float((np.abs(got - ref) / scale).max())


def lu_split(LU):
    """Compact LU -> (L, U) with the unit diagonal of U made explicit."""
    LU = np.asarray(LU, dtype=np.float64)
    L = np.tril(LU)
    U = np.triu(LU, 1) + np.eye(LU.shape[0])
    return L, U


def row_scaled_err(got, ref, u: float) -> float:
    """Error of a computed Cholesky factor in units of its rounding model.

    Entry (i, j) of the factor is an accumulation of j products L_ik L_jk in
    working precision u, divided by L_jj; with rounding errors of random
    sign its error is about u * sqrt(j + 1) times the typical size of the
    entries of row i.  Returns max over the lower triangle of
        |got_ij - ref_ij| / (u * sqrt(j + 1) * rms_i),
    rms_i = ||ref[i, :i+1]||_2 / sqrt(i + 1).  A value of a few units means
    rounding at precision u; a dropped or wrong term gives values of order
    1/u."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    n = ref.shape[0]
    if n == 0:
        return 0.0
    Lr = np.tril(ref)
    rms = np.sqrt((Lr * Lr).sum(1) / np.arange(1, n + 1))
    scale = u * np.sqrt(np.arange(1, n + 1))[None, :] * rms[:, None]
    err = np.tril(np.abs(got - ref)) / np.maximum(scale, 1e-300)
    return float(err.max())
