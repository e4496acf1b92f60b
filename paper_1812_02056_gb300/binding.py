"""ctypes binding of the gbchol C ABI (include/gbchol.h).

Argument marshalling only: every step of every call runs in the CUDA
library.  Each ``gb_*`` function here takes the same arguments as its C
counterpart (pointers as ints); the ``chol_factor`` / ``lu_factor`` /
``chol_solve`` / ``lu_solve`` helpers accept torch tensors (or numpy arrays
for host buffers) and pass their data pointers.

Importing this module loads ``libgbchol.so`` from the package directory and
raises if it is absent: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgbchol.so")

GB_OK = 0
GB_ERR_NOMEM = -1001
GB_ERR_CUDA = -1002
GB_ERR_TIMEOUT = -1003
GB_ERR_NOT_CONVERGED = -1004
GB_ERR_REJECTED = -1005
GB_ERR_UNSUPPORTED = -1006
GB_ERR_BREAKDOWN = -1007
GB_ERR_STATE = -1008

GB_F64, GB_F32, GB_MIX_BF16, GB_MIX_F16, GB_MIX_BF16X3 = 0, 1, 2, 3, 4
DTYPES = {"f64": GB_F64, "f32": GB_F32, "mix_bf16": GB_MIX_BF16, "mix_f16": GB_MIX_F16,
          "mix_bf16x3": GB_MIX_BF16X3}

GB_OPT_INNER_STEP, GB_OPT_USE_GRAPHS, GB_OPT_TC_UPDATE, GB_OPT_SPIN_LIMIT = 1, 2, 3, 4
GB_OPT_PROFILE = 5
GB_OPT_BATCHED_EXACT = 6
GB_OPT_LOOKAHEAD = 7
GB_OPT_STRASSEN = 8
GB_OPT_QR_INNER_STEP = 9
GB_OPT_LEFT_LOOKING = 10
GB_OPT_TEST_WITHHOLD = 11
GB_OPT_INNER_CUDA_CORES = 12
GB_OPT_INNER_RECURSIVE = 13
GB_OPT_INNER_LOOKAHEAD = 14
GB_OPT_EARLY_REST = 15
GB_OPT_RESIDUAL = 16
GB_OPT_F64_UPDATE = 17
PEAKS = {"dfma": 0, "ffma": 1, "dmma": 2, "tc_bf16": 3, "tc_f16": 4, "tc_tf32": 5,
         "dfma_dmma": 6}


class GbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: status {status} ({status_string(status)}) {last_error()}")


class RefineOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nrhs", ctypes.c_int64), ("dtype", ctypes.c_int),
                ("s", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("X", ctypes.c_void_p),
                ("ldx", ctypes.c_int64), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("info", ctypes.c_int), ("iterations", ctypes.c_int),
                ("eta", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("compute_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("running", ctypes.c_int),
                ("max_running", ctypes.c_int), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("budget_bytes", ctypes.c_size_t),
                ("bytes_in_use", ctypes.c_size_t)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("eta", ctypes.c_double)]


# (name, restype, argtypes) of every exported symbol declared in gbchol.h
_I64, _I32, _P, _D = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
SIGNATURES = {
    "gb_status_string": (ctypes.c_char_p, [_I32]),
    "gb_version": (_I32, []),
    "gb_last_error": (ctypes.c_char_p, []),
    "gb_create": (_I32, [ctypes.POINTER(_P), _I32]),
    "gb_destroy": (_I32, [_P]),
    "gb_set_option": (_I32, [_P, _I32, _I64]),
    "gb_get_option": (_I32, [_P, _I32, ctypes.POINTER(_I64)]),
    "gb_chol_factor": (_I32, [_P, _I64, _I64, _I32, _P, _I64, _P, _I64, _P, _P]),
    "gb_lu_factor": (_I32, [_P, _I64, _I64, _I32, _P, _I64, _P, _I64, _P, _P]),
    "gb_qr_factor": (_I32, [_P, _I64, _I64, _I32, _P, _I64, _P, _I64, _P, _I64, _P, _P]),
    "gb_tune_step": (_I32, [_P, _I32, _I32, _I64, _P, _P, _P]),
    "gb_chol_solve": (_I32, [_P, _I64, _I64, _I32, _P, _I64, _P, _I64, _P, _I64, _P, _I64,
                             ctypes.POINTER(RefineOpts), ctypes.POINTER(SolveStats), _P]),
    "gb_lu_solve": (_I32, [_P, _I64, _I64, _I32, _P, _I64, _P, _I64, _P, _I64, _P, _I64,
                           ctypes.POINTER(RefineOpts), ctypes.POINTER(SolveStats), _P]),
    "gb_backward_error": (_I32, [_P, _I32, _I64, _I32, _P, _I64, _P, _I64,
                                 ctypes.POINTER(_D), _P]),
    "gb_residual": (_I32, [_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64,
                           ctypes.POINTER(_D), _P]),
    "gb_chol_factor_batched": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _I32, _I64, _P, _P]),
    "gb_batched_plan": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _I32, _I64, _P]),
    "gb_lu_factor_batched": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _I32, _I64, _P, _P]),
    "gb_lu_batched_plan": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _I32, _I64, _P]),
    "gb_batched_run": (_I32, [_P, _P, _P]),
    "gb_chol_solve_noalloc": (_I32, [_I64, _I64, _I32, _P, _I64, _P, _I64, _P, _I64, _P]),
    "gb_rank_update": (_I32, [_P, _I32, _I32, _I32, _I64, _I64, _I64, _P, _I64, _P, _I64, _P,
                              _I64, _P]),
    "gb_batched_tune": (_I32, [_P, _I32, _I64, _P, _P]),
    "gb_server_create": (_I32, [_I32, ctypes.c_size_t, _I32, ctypes.POINTER(_P)]),
    "gb_server_submit": (_I32, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "gb_server_wait": (_I32, [_P, ctypes.c_uint64, _D, ctypes.POINTER(Result)]),
    "gb_server_poll": (_I32, [_P, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "gb_server_get_stats": (_I32, [_P, ctypes.POINTER(ServerStats)]),
    "gb_server_reset_stats": (_I32, [_P]),
    "gb_server_destroy": (_I32, [_P]),
    "gb_profile_read": (_I32, [_P, _P]),
    "gb_kernel_launches": (ctypes.c_uint64, []),
    "gb_measure_fma_peak": (_I32, [_P, _I32, ctypes.POINTER(_D)]),
    "gb_measure_peak": (_I32, [_P, _I32, ctypes.POINTER(_D)]),
}

PHASES = ["copy", "diag", "panel", "inner", "update"]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 5), ("ms", ctypes.c_double * 5),
                ("flops", ctypes.c_double * 5), ("bytes", ctypes.c_double * 5)]

    def as_dict(self):
        return {p: {"launches": int(self.launches[i]), "ms": float(self.ms[i]),
                    "flops": float(self.flops[i]), "bytes": float(self.bytes[i])}
                for i, p in enumerate(PHASES)}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (once) and declare every entry point's signature."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(
                f"gbchol CUDA library not found at {path}; build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def gb_chol_solve_noalloc(n, nrhs, dt, L, ldl, B, ldb, X, ldx, stream=None) -> int:
    """Solve without a handle or any allocation (include/gbchol.h)."""
    return load().gb_chol_solve_noalloc(n, nrhs, dt, _ptr(L), ldl, _ptr(B), ldb, _ptr(X), ldx,
                                        _stream_ptr(stream))


def kernel_launches() -> int:
    return int(load().gb_kernel_launches())


def status_string(st: int) -> str:
    return load().gb_status_string(int(st)).decode()


def last_error() -> str:
    return load().gb_last_error().decode()


def check(st: int, where: str) -> int:
    if st != GB_OK:
        raise GbError(st, where)
    return st


def _ptr(x) -> int | None:
    """Data pointer of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _ld(x) -> int:
    if hasattr(x, "stride") and callable(x.stride):
        return int(x.stride(0))
    return int(x.strides[0] // x.itemsize)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Handle:
    """Owns a ``gb_handle`` for one device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        check(self.lib.gb_create(ctypes.byref(h), int(device)), "gb_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.gb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, opt: int, value: int):
        check(self.lib.gb_set_option(self.h, int(opt), int(value)), "gb_set_option")

    def get_option(self, opt: int) -> int:
        v = ctypes.c_int64()
        check(self.lib.gb_get_option(self.h, int(opt), ctypes.byref(v)), "gb_get_option")
        return v.value

    def profile_read(self, into=None):
        p = into if into is not None else Profile()
        check(self.lib.gb_profile_read(self.h, ctypes.byref(p)), "gb_profile_read")
        return p

    def measure_peak(self, kind: str) -> float:
        """Measured pipe peak in flop/s: dfma, ffma, dmma, tc_bf16, tc_f16, tc_tf32."""
        v = ctypes.c_double()
        check(self.lib.gb_measure_peak(self.h, PEAKS[kind], ctypes.byref(v)), "gb_measure_peak")
        return v.value

    def measure_fma_peak(self, dtype: str = "f64") -> float:
        v = ctypes.c_double()
        check(self.lib.gb_measure_fma_peak(self.h, DTYPES[dtype], ctypes.byref(v)),
              "gb_measure_fma_peak")
        return v.value

    # ------------------------------------------------------------ raw calls
    def gb_chol_factor(self, n, s, dt, A, lda, L, ldl, info, stream=None) -> int:
        return self.lib.gb_chol_factor(self.h, n, s, dt, _ptr(A), lda, _ptr(L), ldl, _ptr(info),
                                       _stream_ptr(stream))

    def gb_lu_factor(self, n, s, dt, A, lda, LU, ldlu, info, stream=None) -> int:
        return self.lib.gb_lu_factor(self.h, n, s, dt, _ptr(A), lda, _ptr(LU), ldlu, _ptr(info),
                                     _stream_ptr(stream))

    def tune_step(self, kind: str, dtype: str, n: int, stream=None):
        """Autotune (s, inner step) for ``kind`` in {"chol", "lu", "qr"} at
        order ``n``; returns the pair, which later ``s = 0`` calls use."""
        kinds = {"chol": 0, "lu": 1, "qr": 2}
        s_out, b_out = ctypes.c_int64(), ctypes.c_int64()
        check(self.lib.gb_tune_step(self.h, kinds[kind], DTYPES[dtype], int(n), ctypes.byref(s_out),
                                    ctypes.byref(b_out), _stream_ptr(stream)), "gb_tune_step")
        return s_out.value, b_out.value

    def gb_qr_factor(self, n, s, dt, A, lda, Q, ldq, R, ldr, info, stream=None) -> int:
        return self.lib.gb_qr_factor(self.h, n, s, dt, _ptr(A), lda, _ptr(Q), ldq, _ptr(R), ldr,
                                     _ptr(info), _stream_ptr(stream))

    def _solve(self, fn, n, nrhs, dt, F, ldf, A, lda, B, ldb, X, ldx, tol, max_iter, stream):
        opts = RefineOpts(tol, max_iter)
        stats = SolveStats()
        st = fn(self.h, n, nrhs, dt, _ptr(F), ldf, _ptr(A), lda, _ptr(B), ldb, _ptr(X), ldx,
                ctypes.byref(opts), ctypes.byref(stats), _stream_ptr(stream))
        return st, stats

    def gb_chol_solve(self, n, nrhs, dt, L, ldl, A, lda, B, ldb, X, ldx, tol=1e-14, max_iter=30,
                      stream=None):
        return self._solve(self.lib.gb_chol_solve, n, nrhs, dt, L, ldl, A, lda, B, ldb, X, ldx,
                           tol, max_iter, stream)

    def gb_lu_solve(self, n, nrhs, dt, LU, ldlu, A, lda, B, ldb, X, ldx, tol=1e-14, max_iter=30,
                    stream=None):
        return self._solve(self.lib.gb_lu_solve, n, nrhs, dt, LU, ldlu, A, lda, B, ldb, X, ldx,
                           tol, max_iter, stream)

    def gb_backward_error(self, is_lu, n, dt, A, lda, F, ldf, stream=None) -> float:
        out = ctypes.c_double()
        check(self.lib.gb_backward_error(self.h, int(is_lu), n, dt, _ptr(A), lda, _ptr(F), ldf,
                                         ctypes.byref(out), _stream_ptr(stream)),
              "gb_backward_error")
        return out.value

    def gb_residual(self, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, stream=None) -> float:
        """R = B - A X (device buffers); returns the normwise backward error."""
        out = ctypes.c_double()
        check(self.lib.gb_residual(self.h, n, nrhs, _ptr(A), lda, _ptr(X), ldx, _ptr(B), ldb,
                                   _ptr(R), ldr, ctypes.byref(out), _stream_ptr(stream)),
              "gb_residual")
        return out.value

    def gb_chol_factor_batched(self, count, n_arr, a_arr, lda_arr, l_arr, ldl_arr, dt, s, info,
                               stream=None):
        return self.lib.gb_chol_factor_batched(self.h, count, _ptr(n_arr), _ptr(a_arr),
                                               _ptr(lda_arr), _ptr(l_arr), _ptr(ldl_arr), dt, s,
                                               _ptr(info), _stream_ptr(stream))

    def gb_batched_plan(self, count, n_arr, a_arr, lda_arr, l_arr, ldl_arr, dt, s, stream=None):
        return self.lib.gb_batched_plan(self.h, count, _ptr(n_arr), _ptr(a_arr), _ptr(lda_arr),
                                        _ptr(l_arr), _ptr(ldl_arr), dt, s, _stream_ptr(stream))

    def gb_lu_factor_batched(self, count, n_arr, a_arr, lda_arr, lu_arr, ldlu_arr, dt, s, info,
                             stream=None):
        return self.lib.gb_lu_factor_batched(self.h, count, _ptr(n_arr), _ptr(a_arr),
                                             _ptr(lda_arr), _ptr(lu_arr), _ptr(ldlu_arr), dt, s,
                                             _ptr(info), _stream_ptr(stream))

    def gb_lu_batched_plan(self, count, n_arr, a_arr, lda_arr, lu_arr, ldlu_arr, dt, s,
                           stream=None):
        return self.lib.gb_lu_batched_plan(self.h, count, _ptr(n_arr), _ptr(a_arr), _ptr(lda_arr),
                                           _ptr(lu_arr), _ptr(ldlu_arr), dt, s,
                                           _stream_ptr(stream))

    def gb_batched_run(self, info, stream=None):
        return self.lib.gb_batched_run(self.h, _ptr(info), _stream_ptr(stream))

    def gb_batched_tune(self, dt, n_max, steps_out=None, stream=None):
        return self.lib.gb_batched_tune(self.h, dt, n_max, _ptr(steps_out), _stream_ptr(stream))

    def chol_factor_batched(self, mats, s: int = 0, dtype: str = "f64", outs=None, stream=None):
        """Factor a list of square CUDA tensors (in place unless `outs` is
        given) in one launch; returns the per-matrix info as a numpy array."""
        return self._factor_batched(self.gb_chol_factor_batched, "gb_chol_factor_batched", mats,
                                    s, dtype, outs, stream)

    def lu_factor_batched(self, mats, s: int = 0, dtype: str = "f64", outs=None, stream=None):
        """Batched Algorithm 2: compact LU of each square CUDA tensor (in place
        unless `outs` is given); returns the per-matrix info."""
        return self._factor_batched(self.gb_lu_factor_batched, "gb_lu_factor_batched", mats, s,
                                    dtype, outs, stream)

    def _factor_batched(self, fn, name, mats, s, dtype, outs, stream):
        import numpy as np
        import torch
        cnt = len(mats)
        outs = mats if outs is None else outs
        n_arr = np.array([m.shape[0] for m in mats], dtype=np.int64)
        a_arr = np.array([m.data_ptr() for m in mats], dtype=np.uint64)
        lda = np.array([max(1, m.stride(0)) for m in mats], dtype=np.int64)
        l_arr = np.array([m.data_ptr() for m in outs], dtype=np.uint64)
        ldl = np.array([max(1, m.stride(0)) for m in outs], dtype=np.int64)
        info = torch.zeros(max(cnt, 1), dtype=torch.int32, device=mats[0].device if mats else "cuda")
        check(fn(cnt, n_arr, a_arr, lda, l_arr, ldl, DTYPES[dtype], s, info, stream), name)
        torch.cuda.synchronize()
        return info[:cnt].cpu().numpy()

    def gb_rank_update(self, dt, lower, y_is_kxn, M, N, K, C, ldc, X, ldx, Y, ldy, stream=None):
        return self.lib.gb_rank_update(self.h, dt, int(lower), int(y_is_kxn), M, N, K, _ptr(C), ldc,
                                       _ptr(X), ldx, _ptr(Y), ldy, _stream_ptr(stream))

    # --------------------------------------------------- tensor conveniences
    def chol_factor(self, A, s: int, dtype: str = "f64", out=None, stream=None):
        """Factor a CUDA (or host) tensor ``A``; returns ``(L, info)``."""
        import torch
        n = A.shape[0]
        dt = DTYPES[dtype]
        ltype = torch.float64 if dt == GB_F64 else torch.float32
        L = out if out is not None else torch.empty((n, n), dtype=ltype, device=A.device)
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
        check(self.gb_chol_factor(n, s, dt, A, _ld(A) if n else 1, L, _ld(L) if n else 1, info,
                                  stream), "gb_chol_factor")
        return L, info

    def lu_factor(self, A, s: int, dtype: str = "f64", out=None, stream=None):
        """Compact LU of ``A``; returns ``(LU, info)``."""
        import torch
        n = A.shape[0]
        dt = DTYPES[dtype]
        ltype = torch.float64 if dt == GB_F64 else torch.float32
        LU = out if out is not None else torch.empty((n, n), dtype=ltype, device=A.device)
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
        check(self.gb_lu_factor(n, s, dt, A, _ld(A) if n else 1, LU, _ld(LU) if n else 1, info,
                                stream), "gb_lu_factor")
        return LU, info

    def qr_factor(self, A, s: int, dtype: str = "f64", stream=None):
        """Algorithm 3: ``A = Q R``; returns ``(Q, R, info)``."""
        import torch
        n = A.shape[0]
        dt = DTYPES[dtype]
        ttype = torch.float64 if dt == GB_F64 else torch.float32
        Q = torch.empty((n, n), dtype=ttype, device=A.device)
        R = torch.empty((n, n), dtype=ttype, device=A.device)
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
        check(self.gb_qr_factor(n, s, dt, A, _ld(A) if n else 1, Q, _ld(Q) if n else 1, R,
                                _ld(R) if n else 1, info, stream), "gb_qr_factor")
        return Q, R, info

    def chol_solve(self, L, B, dtype: str = "f64", A=None, tol=1e-14, max_iter=30, stream=None,
                   allow_not_converged=False):
        import torch
        n, r = B.shape
        X = torch.empty_like(B)
        st, stats = self.gb_chol_solve(n, r, DTYPES[dtype], L, _ld(L), A,
                                       _ld(A) if A is not None else n, B, _ld(B), X, _ld(X), tol,
                                       max_iter, stream)
        if not (allow_not_converged and st == GB_ERR_NOT_CONVERGED):
            check(st, "gb_chol_solve")
        return X, stats

    def lu_solve(self, LU, B, dtype: str = "f64", A=None, tol=1e-14, max_iter=30, stream=None,
                 allow_not_converged=False):
        import torch
        n, r = B.shape
        X = torch.empty_like(B)
        st, stats = self.gb_lu_solve(n, r, DTYPES[dtype], LU, _ld(LU), A,
                                     _ld(A) if A is not None else n, B, _ld(B), X, _ld(X), tol,
                                     max_iter, stream)
        if not (allow_not_converged and st == GB_ERR_NOT_CONVERGED):
            check(st, "gb_lu_solve")
        return X, stats

    def backward_error(self, A, F, dtype: str = "f64", lu: bool = False, stream=None) -> float:
        n = A.shape[0]
        return self.gb_backward_error(1 if lu else 0, n, DTYPES[dtype], A, _ld(A), F, _ld(F),
                                      stream)


class Server:
    """Continuous-batching factor-and-solve server (gb_server_*)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, max_slots: int = 4):
        self.lib = load()
        p = ctypes.c_void_p()
        check(self.lib.gb_server_create(int(device), int(hbm_budget), int(max_slots),
                                        ctypes.byref(p)), "gb_server_create")
        self.p = p
        self._keep = {}

    def submit(self, A, B, X, dtype: str = "mix_bf16", s: int = 0, tol: float = 1e-14,
               max_iter: int = 30) -> int:
        """Queue A X = B (tensors or arrays stay referenced until waited for)."""
        n, nrhs = B.shape
        r = Request(n, nrhs, DTYPES[dtype], s, _ptr(A), _ld(A), _ptr(B), _ld(B), _ptr(X), _ld(X),
                    tol, max_iter)
        t = ctypes.c_uint64()
        check(self.lib.gb_server_submit(self.p, ctypes.byref(r), ctypes.byref(t)),
              "gb_server_submit")
        self._keep[t.value] = (A, B, X)
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0) -> Result:
        res = Result()
        check(self.lib.gb_server_wait(self.p, ticket, timeout_s, ctypes.byref(res)),
              "gb_server_wait")
        self._keep.pop(ticket, None)
        return res

    def poll(self, ticket: int):
        res = Result()
        st = self.lib.gb_server_poll(self.p, ticket, ctypes.byref(res))
        if st == GB_ERR_STATE:
            return None
        check(st, "gb_server_poll")
        self._keep.pop(ticket, None)
        return res

    def stats(self) -> ServerStats:
        s = ServerStats()
        check(self.lib.gb_server_get_stats(self.p, ctypes.byref(s)), "gb_server_get_stats")
        return s

    def reset_stats(self):
        check(self.lib.gb_server_reset_stats(self.p), "gb_server_reset_stats")

    def close(self):
        if self.p:
            self.lib.gb_server_destroy(self.p)
            self.p = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
