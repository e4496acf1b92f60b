"""gb_chol_solve_noalloc: the solve for callers that cannot allocate.

Callers working inside a memory budget they do not own, in latency-critical
sections where an allocation (which can synchronize the device) is not
allowed, or in a plugin that must not touch its host program's allocator
cannot create a handle (gb_create allocates); this entry point keeps its
scratch in a static device array.  The tests call it through the C ABI,
twice in a row and across changes of n, and check each result against the
regular gb_chol_solve within the solve tolerance of the suite -- 1e-10 of
max |X| for FP64 factors, 1e-5 for FP32 factors (the two entry points reach
X by different, equally valid roundings: substitution here, inverted
diagonal blocks in the regular solve) -- against the CPU oracle's
substitution with the same factor, and by the solve's backward error against
A.  The file is collected last and must pass alone in a fresh process as
well as after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I

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


def _tol(dtype):
    return 1e-10 if dtype == "f64" else 1e-5


def _eta(A, X, B):
    """max over right-hand sides of |b - A x|_inf / (|A|_inf |x|_inf + |b|_inf)."""
    R = B - A @ X
    den = np.abs(A).sum(1).max() * np.abs(X).max(0) + np.abs(B).max(0)
    return float((np.abs(R).max(0) / den).max())


def _factor(h, dtype, n, seed):
    A = I.spd_gram(n, seed)
    tt = torch.float64 if dtype == "f64" else torch.float32
    src = torch.from_numpy(A).to(DEV, torch.float64 if dtype.startswith("mix") else tt)
    L, info = h.chol_factor(src, 64, dtype)
    assert int(info.item()) == 0
    return A, L


def _noalloc(dtype, L, ldl, B, ldb, X, ldx, n, nrhs):
    from paper_1812_02056_gb300 import binding
    st = binding.gb_chol_solve_noalloc(n, nrhs, binding.DTYPES[dtype], L, ldl, B, ldb, X, ldx)
    torch.cuda.synchronize()
    return st


# backward error of a plain substitution with the factor, bounded by the
# factor's own backward error: FP64 and FP32 working precision, or the BF16
# operands of the mixed factor's delayed update (unit roundoff 2^-8)
ETA = {"f64": 1e-14, "f32": 1e-5, "mix_bf16": 1e-2}


def _check(dtype, A, L, B, got, ref, eta_dtype=None):
    tol = _tol(dtype)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    Lo = L.double().cpu().numpy()
    want = oracle.chol_solve(np.tril(Lo), B)
    assert np.abs(got - want).max() <= tol * np.abs(want).max()
    # plain substitution with the factor: backward error at the factor's precision
    assert _eta(A, got, B) <= ETA[eta_dtype or dtype]


@pytest.mark.parametrize("dtype,n,nrhs", [("f64", 1000, 7), ("f32", 777, 33)])
def test_noalloc_solve_matches_regular_solve_twice(h, dtype, n, nrhs):
    from paper_1812_02056_gb300 import binding
    A, L = _factor(h, dtype, n, 4242 + n)
    Bn = I.rhs(n, nrhs, 99)
    B = torch.from_numpy(Bn).to(DEV)
    X_ref, _ = h.chol_solve(L, B, dtype)
    ref = X_ref.cpu().numpy()
    for _ in range(2):
        X = torch.full_like(B, float("nan"))
        st = _noalloc(dtype, L, L.stride(0), B, nrhs, X, nrhs, n, nrhs)
        assert st == binding.GB_OK, binding.status_string(st)
        _check(dtype, A, L, Bn, X.cpu().numpy(), ref)


def test_noalloc_mixed_factor_float_l(h):
    """A GB_MIX_BF16 factor is float: the call reads L as float."""
    from paper_1812_02056_gb300 import binding
    n, nrhs = 513, 5
    A, L = _factor(h, "mix_bf16", n, 7001)
    assert L.dtype == torch.float32
    Bn = I.rhs(n, nrhs, 98)
    B = torch.from_numpy(Bn).to(DEV)
    X_ref, _ = h.chol_solve(L, B, "mix_bf16")
    X = torch.empty_like(B)
    assert _noalloc("mix_bf16", L, n, B, nrhs, X, nrhs, n, nrhs) == binding.GB_OK
    _check("f32", A, L, Bn, X.cpu().numpy(), X_ref.cpu().numpy(), eta_dtype="mix_bf16")


def test_noalloc_in_place_and_padded_leading_dimensions(h):
    """X == B (in place), ldl > n and ldx > nrhs."""
    from paper_1812_02056_gb300 import binding
    n, nrhs, pad_l, pad_x = 300, 3, 17, 5
    A, L = _factor(h, "f64", n, 7002)
    Lp = torch.full((n, n + pad_l), float("nan"), dtype=torch.float64, device=DEV)
    Lp[:, :n] = L
    Bn = I.rhs(n, nrhs, 97)
    X_ref, _ = h.chol_solve(L, torch.from_numpy(Bn).to(DEV), "f64")
    XB = torch.full((n, nrhs + pad_x), -7.0, dtype=torch.float64, device=DEV)
    XB[:, :nrhs] = torch.from_numpy(Bn).to(DEV)
    ld = nrhs + pad_x
    assert _noalloc("f64", Lp, n + pad_l, XB, ld, XB, ld, n, nrhs) == binding.GB_OK
    got = XB.cpu().numpy()
    assert np.all(got[:, nrhs:] == -7.0)  # the padding is not touched
    _check("f64", A, L, Bn, got[:, :nrhs], X_ref.cpu().numpy())


def test_noalloc_changing_order_between_calls(h):
    """Back-to-back calls of different n reuse the shared flags under new
    epochs: a large solve, a small one, then the large one again."""
    from paper_1812_02056_gb300 import binding
    cases = []
    for n in (2048, 100, 2048, 33):
        A, L = _factor(h, "f64", n, 7100 + n)
        Bn = I.rhs(n, 4, 96 + n)
        B = torch.from_numpy(Bn).to(DEV)
        X_ref, _ = h.chol_solve(L, B, "f64")
        cases.append((A, L, Bn, B, X_ref.cpu().numpy()))
    for A, L, Bn, B, ref in cases:
        n = L.shape[0]
        X = torch.full_like(B, float("nan"))
        assert _noalloc("f64", L, n, B, 4, X, 4, n, 4) == binding.GB_OK
        _check("f64", A, L, Bn, X.cpu().numpy(), ref)


def test_noalloc_breakdown_then_recovers(h):
    """A zero diagonal entry returns GB_ERR_BREAKDOWN; the next call with a
    good factor succeeds (the breakdown word is cleared per call)."""
    from paper_1812_02056_gb300 import binding
    n = 200
    A, L = _factor(h, "f64", n, 7003)
    bad = L.clone()
    bad[77, 77] = 0.0
    Bn = I.rhs(n, 2, 95)
    B = torch.from_numpy(Bn).to(DEV)
    X = torch.empty_like(B)
    assert _noalloc("f64", bad, n, B, 2, X, 2, n, 2) == binding.GB_ERR_BREAKDOWN
    bad[77, 77] = float("nan")
    assert _noalloc("f64", bad, n, B, 2, X, 2, n, 2) == binding.GB_ERR_BREAKDOWN
    X_ref, _ = h.chol_solve(L, B, "f64")
    assert _noalloc("f64", L, n, B, 2, X, 2, n, 2) == binding.GB_OK
    _check("f64", A, L, Bn, X.cpu().numpy(), X_ref.cpu().numpy())


def test_noalloc_rejects_beyond_maximum_and_host_buffers(h):
    from paper_1812_02056_gb300 import binding
    d = torch.zeros(4, dtype=torch.float64, device=DEV)
    st = binding.gb_chol_solve_noalloc(131073, 1, binding.GB_F64, d, 131073, d, 1, d, 1)
    assert st == binding.GB_ERR_UNSUPPORTED
    Lh = np.eye(8)
    Bh = np.ones((8, 1))
    Xd = torch.zeros((8, 1), dtype=torch.float64, device=DEV)
    assert binding.gb_chol_solve_noalloc(8, 1, binding.GB_F64, Lh, 8, Bh, 1, Xd, 1) == -4
    Ld = torch.eye(8, dtype=torch.float64, device=DEV)
    assert binding.gb_chol_solve_noalloc(8, 1, binding.GB_F64, Ld, 8, Bh, 1, Xd, 1) == -6
    Xh = np.zeros((8, 1))
    Bd = torch.ones((8, 1), dtype=torch.float64, device=DEV)
    assert binding.gb_chol_solve_noalloc(8, 1, binding.GB_F64, Ld, 8, Bd, 1, Xh, 1) == -8
    if torch.cuda.device_count() > 1:
        # another GPU's memory is rejected before any launch
        Lo = torch.eye(8, dtype=torch.float64, device="cuda:1")
        assert binding.gb_chol_solve_noalloc(8, 1, binding.GB_F64, Lo, 8, Bd, 1, Bd, 1) == -4
