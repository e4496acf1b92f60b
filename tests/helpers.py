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
