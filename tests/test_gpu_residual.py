"""The residual r = b - A x of FP64 refinement (`gb_residual`, the step that
brings the low-precision solves back to FP64 accuracy) by both methods of
GB_OPT_RESIDUAL: FP64 multiply-adds on the CUDA cores (0) and exact digit
products on the tensor cores (1).

* Integer A, x, b whose products and sums are exact in FP64: both methods
  give the exact residual, bit for bit (ragged orders, K split over CTAs,
  and an order above the 2^14 terms one exact FP32 accumulation can take).
* Random A (the refinement workloads' SPD matrices) and x with a spread of
  magnitudes, against the correctly rounded residual (exact products by
  Veltkamp splitting, summed by math.fsum): the digit method errs by less
  than 2^-48 sigma_i tau_c, sigma_i and tau_c being the powers of two that
  scale row i of A and column c of x.  Dropping the smallest digit pairs
  kept, or one digit plane, errs by 2^-44 sigma_i tau_c or more.
* Refinement with either method converges to eta <= 1e-14 and matches the
  oracle's FP64 solve.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests.helpers import exact_dot_minus, pow2_scale

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


def _t(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _residual(h, method, A, X, B):
    from paper_1812_02056_gb300 import binding
    n, nrhs = X.shape
    R = torch.full((n, nrhs), float("nan"), dtype=torch.float64, device=DEV)
    prev = h.get_option(binding.GB_OPT_RESIDUAL)
    h.set_option(binding.GB_OPT_RESIDUAL, method)
    try:
        eta = h.gb_residual(n, nrhs, A, A.shape[1], X, nrhs, B, nrhs, R, nrhs)
    finally:
        h.set_option(binding.GB_OPT_RESIDUAL, prev)
    return R.cpu().numpy(), eta


@pytest.mark.parametrize("n,nrhs", [(300, 3), (2100, 16), (5000, 23)])
@pytest.mark.parametrize("method", [0, 1])
def test_integer_residual_is_exact(h, n, nrhs, method):
    rng = np.random.default_rng(n + nrhs)
    A = rng.integers(-1000, 1001, (n, n))
    X = rng.integers(-1000, 1001, (n, nrhs))
    B = rng.integers(-10 ** 6, 10 ** 6 + 1, (n, nrhs))
    ref = (B - A @ X).astype(np.float64)  # int64: exact
    R, eta = _residual(h, method, _t(A), _t(X), _t(B))
    assert np.array_equal(R, ref)
    den = np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0)
    assert eta == pytest.approx((np.abs(ref).max(0) / den).max(), rel=1e-14)


def test_digit_method_beyond_one_exact_accumulation(h):
    """n = 17500 > 2^14 with every digit at its largest (1023 = 0.1111111111b
    x 2^10): one FP32 accumulation over all of K would pass 2^24, so the
    product runs over two K ranges; the result stays exact."""
    n, nrhs = 17500, 2
    A = torch.full((n, n), 1023.0, dtype=torch.float64, device=DEV)
    A[1::3] = 1022.0
    X = torch.full((n, nrhs), 1023.0, dtype=torch.float64, device=DEV)
    X[:, 1] = -1021.0
    B = torch.zeros((n, nrhs), dtype=torch.float64, device=DEV)
    R, _ = _residual(h, 1, A, X, B)
    rows = np.where(np.arange(n) % 3 == 1, 1022, 1023).astype(np.int64)
    ref = -(rows[:, None] * n * np.array([1023, -1021], dtype=np.int64)[None, :])
    assert np.array_equal(R, ref.astype(np.float64))
    del A


@pytest.mark.parametrize("n,nrhs", [(3000, 16), (4500, 5)])
def test_digit_method_against_correctly_rounded_residual(h, n, nrhs):
    A = I.spd_logspaced(n, 21, cond=1e4)
    rng = np.random.default_rng(22)
    X = I.rhs(n, nrhs, 23) * 10.0 ** rng.uniform(-3, 3, (n, nrhs))
    B = I.rhs(n, nrhs, 24)
    Ad, Xd, Bd = _t(A), _t(X), _t(B)
    Rs, eta_s = _residual(h, 1, Ad, Xd, Bd)
    Rf, eta_f = _residual(h, 0, Ad, Xd, Bd)
    rows = sorted({0, 1, n // 3, n // 2, n - 2, n - 1, *rng.integers(0, n, 10).tolist()})
    worst_s = worst_f = 0.0
    for i in rows:
        sig = pow2_scale(A[i])
        for c in range(nrhs):
            ref = exact_dot_minus(B[i, c], A[i], X[:, c])
            scale = sig * pow2_scale(X[:, c])
            worst_s = max(worst_s, abs(Rs[i, c] - ref) / scale)
            worst_f = max(worst_f, abs(Rf[i, c] - ref) / scale)
    assert worst_s <= 2.0 ** -48, (worst_s, worst_f)
    assert worst_f <= n * 2.0 ** -52
    # the reported eta: the same up to the residuals' own error
    assert eta_s == pytest.approx(eta_f, rel=1e-10)


@pytest.mark.parametrize("method", [0, 1])
def test_residual_non_finite_gives_infinite_eta(h, method):
    n, nrhs = 2100, 3
    A = I.spd_gram(n, 5)
    X = I.rhs(n, nrhs, 6)
    B = I.rhs(n, nrhs, 7)
    A2 = A.copy()
    A2[5, 17] = np.nan
    _, eta = _residual(h, method, _t(A2), _t(X), _t(B))
    assert eta == math.inf
    X2 = X.copy()
    X2[40, 1] = np.inf
    _, eta = _residual(h, method, _t(A), _t(X2), _t(B))
    assert eta == math.inf


def test_residual_option_and_arguments(h):
    from paper_1812_02056_gb300 import binding
    assert h.get_option(binding.GB_OPT_RESIDUAL) == 2  # the default: digits from n = 2048
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_RESIDUAL, 3) == -3
    n = 64
    A = _t(np.eye(n))
    X = torch.ones((n, 2), dtype=torch.float64, device=DEV)
    R = torch.empty_like(X)
    import ctypes
    eta = ctypes.c_double()
    lib = h.lib
    host = np.ones((n, 2))
    assert lib.gb_residual(h.h, n, 2, host.ctypes.data, n, X.data_ptr(), 2, X.data_ptr(), 2,
                           R.data_ptr(), 2, ctypes.byref(eta), None) == -4
    assert lib.gb_residual(h.h, n, 2, A.data_ptr(), n, X.data_ptr(), 2, X.data_ptr(), 2,
                           R.data_ptr(), 1, ctypes.byref(eta), None) == -11
    assert lib.gb_residual(h.h, 0, 2, None, 1, None, 2, None, 2, None, 2, ctypes.byref(eta),
                           None) == 0


@pytest.mark.parametrize("method", [0, 1])
def test_refinement_with_either_residual(h, method):
    from paper_1812_02056_gb300 import binding
    n, nrhs = 2500, 16
    A = I.spd_logspaced(n, 31, cond=1e4)
    B = I.rhs(n, nrhs, 32)
    Ad = _t(A)
    L, info = h.chol_factor(Ad, 256, "mix_bf16x3")
    assert int(info.item()) == 0
    prev = h.get_option(binding.GB_OPT_RESIDUAL)
    h.set_option(binding.GB_OPT_RESIDUAL, method)
    try:
        X, stats = h.chol_solve(L, _t(B), "mix_bf16x3", A=Ad, tol=1e-14, max_iter=20)
    finally:
        h.set_option(binding.GB_OPT_RESIDUAL, prev)
    assert stats.converged == 1 and stats.eta <= 1e-14
    Xg = X.cpu().numpy()
    Lo, _ = oracle.chol(A, 256)
    Xo = oracle.chol_solve(Lo, B)
    assert np.abs(Xg - Xo).max() <= 1e4 * 1e-13 * np.abs(Xo).max()
    R = B - A @ Xg
    eta = max(np.abs(R[:, c]).max() / (np.abs(A).sum(1).max() * np.abs(Xg[:, c]).max()
                                        + np.abs(B[:, c]).max()) for c in range(nrhs))
    assert eta <= 2e-14


def test_lu_refinement_with_digit_residual(h):
    from paper_1812_02056_gb300 import binding
    n, nrhs = 2100, 4
    A = I.lu_diag_dominant(n, 41)
    B = I.rhs(n, nrhs, 42)
    LU, info = h.lu_factor(_t(A, torch.float32), 256, "f32")
    assert int(info.item()) == 0
    h.set_option(binding.GB_OPT_RESIDUAL, 1)
    try:
        X, stats = h.lu_solve(LU, _t(B), "f32", A=_t(A), tol=1e-15)
    finally:
        h.set_option(binding.GB_OPT_RESIDUAL, 2)
    assert stats.converged == 1 and stats.eta <= 1e-15
    Xo = np.linalg.solve(A, B)
    assert np.abs(X.cpu().numpy() - Xo).max() <= 1e-12 * np.abs(Xo).max()
