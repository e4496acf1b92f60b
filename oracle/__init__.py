"""Plain FP64 CPU oracle for Algorithms 1, 2 and 3 of arXiv:1812.02056.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it to check and to time the CUDA library.
The library itself never imports it.

The arithmetic lives in ``oracle.c`` (C, FP64, compiled with
``-O2 -ffp-contract=off``); this module compiles it with gcc on first use and
wraps it with numpy arrays.  Each wrapper cites the part of the paper it
follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

FULL_SQUARE = 1
SEQUENTIAL = 2

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        P = ctypes.c_void_p
        lib.orc_chol.argtypes = [i64, i64, P, i64, P, i64, i32]
        lib.orc_chol.restype = i64
        lib.orc_lu.argtypes = [i64, i64, P, i64, P, i64, P, i64, i32]
        lib.orc_lu.restype = i64
        lib.orc_qr.argtypes = [i64, i64, P, i64, P, i64, P, i64, i32]
        lib.orc_qr.restype = i64
        lib.orc_qr_backward_error.argtypes = [i64, P, i64, P, i64, P, i64]
        lib.orc_qr_backward_error.restype = dbl
        lib.orc_orthogonality.argtypes = [i64, P, i64]
        lib.orc_orthogonality.restype = dbl
        for name in ("orc_solve_lower", "orc_solve_lower_trans", "orc_solve_unit_upper",
                     "orc_chol_solve"):
            getattr(lib, name).argtypes = [i64, i64, P, i64, P, i64]
            getattr(lib, name).restype = None
        lib.orc_lu_solve.argtypes = [i64, i64, P, i64, P, i64, P, i64]
        lib.orc_lu_solve.restype = None
        lib.orc_residual.argtypes = [i64, i64, P, i64, P, i64, P, i64, P, i64]
        lib.orc_residual.restype = None
        lib.orc_chol_refine.argtypes = [i64, i64, P, i64, P, i64, P, i64, P, i64, dbl, i64,
                                        ctypes.POINTER(dbl)]
        lib.orc_chol_refine.restype = i64
        lib.orc_chol_backward_error.argtypes = [i64, P, i64, P, i64]
        lib.orc_chol_backward_error.restype = dbl
        lib.orc_lu_backward_error.argtypes = [i64, P, i64, P, i64, P, i64]
        lib.orc_lu_backward_error.restype = dbl
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = i32
        lib.orc_set_num_threads.argtypes = [i32]
        lib.orc_set_num_threads.restype = None
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(t: int) -> None:
    _load().orc_set_num_threads(int(t))


def chol(A, s: int, full_square: bool = False, sequential: bool = False):
    """Algorithm 1 (fast Cholesky, step ``s``).  Returns ``(L, info)``:
    ``info`` is 0, or ``c+1`` (1-based column) at the first non-positive
    pivot.  Reads the lower triangle of ``A`` unless ``full_square``."""
    A = _f64(A)
    n = A.shape[0]
    L = np.zeros((n, n))
    mode = (FULL_SQUARE if full_square else 0) | (SEQUENTIAL if sequential else 0)
    info = _load().orc_chol(n, int(s), _p(A), n, _p(L), n, mode)
    if info < 0:
        raise ValueError(f"orc_chol failed ({info})")
    return L, int(info)


def lu(A, s: int, sequential: bool = False):
    """Algorithm 2 (fast LU, step ``s``, no pivoting): ``A = L U`` with ``U``
    unit upper triangular.  Returns ``(L, U, info)``."""
    A = _f64(A)
    n = A.shape[0]
    L = np.zeros((n, n))
    U = np.zeros((n, n))
    mode = SEQUENTIAL if sequential else 0
    info = _load().orc_lu(n, int(s), _p(A), n, _p(L), n, _p(U), n, mode)
    if info < 0:
        raise ValueError(f"orc_lu failed ({info})")
    return L, U, int(info)


def qr(A, s: int, full_r: bool = False):
    """Algorithm 3 (fast QR, step ``s``, block Gram-Schmidt): ``A = Q R``.
    Returns ``(Q, R, info)``; ``R`` is the upper triangle of ``Q^T A`` (all of
    it with ``full_r``)."""
    A = _f64(A)
    n = A.shape[0]
    Q = np.zeros((n, n))
    R = np.zeros((n, n))
    mode = FULL_SQUARE if full_r else 0
    info = _load().orc_qr(n, int(s), _p(A), n, _p(Q), n, _p(R), n, mode)
    if info < 0:
        raise ValueError(f"orc_qr failed ({info})")
    return Q, R, int(info)


def qr_backward_error(A, Q, R) -> float:
    """``||A - Q R||_F / ||A||_F`` in long double."""
    A, Q, R = _f64(A), _f64(Q), _f64(R)
    return float(_load().orc_qr_backward_error(A.shape[0], _p(A), A.shape[0], _p(Q), Q.shape[0],
                                               _p(R), R.shape[0]))


def orthogonality(Q) -> float:
    """``||Q^T Q - I||_F`` in long double."""
    Q = _f64(Q)
    return float(_load().orc_orthogonality(Q.shape[0], _p(Q), Q.shape[0]))


def _rhs(B):
    B = _f64(B)
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None].copy()
    return B, squeeze


def chol_solve(L, B):
    """``X = (L L^T)^{-1} B`` by forward then back substitution."""
    L = _f64(L)
    X, squeeze = _rhs(np.array(B, dtype=np.float64, copy=True))
    _load().orc_chol_solve(L.shape[0], X.shape[1], _p(L), L.shape[0], _p(X), X.shape[1])
    return X[:, 0] if squeeze else X


def lu_solve(L, U, B):
    """``X = (L U)^{-1} B``, ``U`` unit upper."""
    L, U = _f64(L), _f64(U)
    X, squeeze = _rhs(np.array(B, dtype=np.float64, copy=True))
    n = L.shape[0]
    _load().orc_lu_solve(n, X.shape[1], _p(L), n, _p(U), n, _p(X), X.shape[1])
    return X[:, 0] if squeeze else X


def solve_lower(L, B, trans: bool = False):
    L = _f64(L)
    X, squeeze = _rhs(np.array(B, dtype=np.float64, copy=True))
    fn = _load().orc_solve_lower_trans if trans else _load().orc_solve_lower
    fn(L.shape[0], X.shape[1], _p(L), L.shape[0], _p(X), X.shape[1])
    return X[:, 0] if squeeze else X


def solve_unit_upper(U, B):
    U = _f64(U)
    X, squeeze = _rhs(np.array(B, dtype=np.float64, copy=True))
    _load().orc_solve_unit_upper(U.shape[0], X.shape[1], _p(U), U.shape[0], _p(X), X.shape[1])
    return X[:, 0] if squeeze else X


def residual(A, X, B):
    """``R = B - A X``."""
    A = _f64(A)
    X, sq = _rhs(X)
    B, _ = _rhs(B)
    R = np.empty_like(B)
    n, r = B.shape
    _load().orc_residual(n, r, _p(A), n, _p(X), r, _p(B), r, _p(R), r)
    return R[:, 0] if sq else R


def chol_refine(A, L, B, tol: float = 1e-14, max_iter: int = 30):
    """Iterative refinement of ``A X = B`` from a Cholesky factor ``L`` (held
    in FP64).  Returns ``(X, iterations, eta)``."""
    A, L = _f64(A), _f64(L)
    B, squeeze = _rhs(B)
    n, r = B.shape
    X = np.empty_like(B)
    eta = ctypes.c_double(0.0)
    it = _load().orc_chol_refine(n, r, _p(A), n, _p(L), n, _p(B), r, _p(X), r, float(tol),
                                 int(max_iter), ctypes.byref(eta))
    if it < 0:
        raise MemoryError("orc_chol_refine")
    return (X[:, 0] if squeeze else X), int(it), float(eta.value)


def chol_backward_error(A, L) -> float:
    """``||A - L L^T||_F / ||A||_F`` accumulated in long double."""
    A, L = _f64(A), _f64(L)
    n = A.shape[0]
    return float(_load().orc_chol_backward_error(n, _p(A), n, _p(L), n))


def lu_backward_error(A, L, U) -> float:
    """``||A - L U||_F / ||A||_F`` (unit diagonal of ``U`` implied)."""
    A, L, U = _f64(A), _f64(L), _f64(U)
    n = A.shape[0]
    return float(_load().orc_lu_backward_error(n, _p(A), n, _p(L), n, _p(U), n))
