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


def _veltkamp(a):
    c = 134217729.0 * a  # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def exact_dot_minus(c, a, b) -> float:
    """c - sum_k a_k b_k correctly rounded: every product as the sum of four
    exact FP64 products of 26-bit halves (Veltkamp), all terms summed
    exactly by math.fsum."""
    import math
    ah, al = _veltkamp(np.asarray(a, dtype=np.float64))
    bh, bl = _veltkamp(np.asarray(b, dtype=np.float64))
    terms = np.concatenate([ah * bh, ah * bl, al * bh, al * bl])
    return math.fsum(np.concatenate([[c], -terms]).tolist())


def pow2_scale(v) -> float:
    """The power of two 2^e with max |v| < 2^e (1 for an all-zero v)."""
    import math
    m = float(np.abs(np.asarray(v)).max()) if np.size(v) else 0.0
    return 2.0 ** math.frexp(m)[1] if m > 0 else 1.0
