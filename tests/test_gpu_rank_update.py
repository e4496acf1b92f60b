"""The delayed rank-s update (gb_rank_update): C -= X op(Y).

* Exact cases: small-integer operands make every product and every partial
  sum exact in FP32 (and the 16-bit roundings exact), so the tensor-core and
  CUDA-core kernels must reproduce C - X op(Y) bit for bit; a wrong
  descriptor, swizzle, lane mapping or mask shows up as a wrong entry.
* Rounded cases: random FP32 operands; the reference is the FP64 product of
  the operands rounded to BF16/FP16 (the kernel's inputs), and the allowed
  error is FP32 accumulation, 4e-6 * (|C| + sum_k |x_k y_k|).
* Lower mode leaves the strict upper triangle untouched, bit for bit.
"""
import numpy as np
import pytest

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


def _run(h, dt, lower, kxn, C, X, Y):
    from paper_1812_02056_gb300 import binding
    M, N = C.shape
    K = X.shape[1]
    st = h.gb_rank_update(binding.DTYPES[dt], lower, kxn, M, N, K, C, C.stride(0), X, X.stride(0),
                          Y, Y.stride(0))
    binding.check(st, "gb_rank_update")
    torch.cuda.synchronize()
    return C


def _round16(x, dt):
    if dt == "mix_bf16x3":
        return x.double()  # the split keeps about FP32 accuracy
    if dt == "mix_bf16":
        return x.to(torch.bfloat16).double()
    if dt == "mix_f16":
        return x.to(torch.float16).double()
    return x.double()


def _expected(C, X, Y, kxn, dt):
    Xr, Yr = _round16(X.cpu(), dt), _round16(Y.cpu(), dt)
    P = Xr @ (Yr if kxn else Yr.T)
    Pa = Xr.abs() @ (Yr.abs() if kxn else Yr.abs().T)
    return C.cpu().double() - P, Pa


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3", "f32", "f64"])
@pytest.mark.parametrize("M,N,K,lower,kxn", [
    (300, 300, 117, 1, 0), (129, 129, 16, 1, 0), (520, 520, 1024, 1, 0), (1, 1, 1, 1, 0),
    (200, 520, 64, 0, 1), (384, 256, 200, 0, 1), (77, 333, 1000, 0, 0), (260, 260, 100, 1, 0)])
def test_rank_update_exact_integers(h, dt, M, N, K, lower, kxn):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    tt = torch.float64 if dt == "f64" else torch.float32
    X = torch.randint(-4, 5, (M, K), generator=g).to(tt)
    Y = torch.randint(-4, 5, (K, N) if kxn else (N, K), generator=g).to(tt)
    if lower and M == N:
        Y = X.clone()  # Cholesky: both operands are R
    C0 = torch.randint(-1000, 1000, (M, N), generator=g).to(tt)
    exp, _ = _expected(C0, X, Y, kxn, dt)
    C = _run(h, dt, lower, kxn, C0.to(DEV), X.to(DEV), Y.to(DEV)).cpu().double()
    if lower:
        mask = torch.tril(torch.ones(M, N, dtype=torch.bool))
        assert torch.equal(C[mask], exp[mask])
        assert torch.equal(C[~mask], C0.double()[~mask])
    else:
        assert torch.equal(C, exp)


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
@pytest.mark.parametrize("M,N,K,lower,kxn", [(1000, 1000, 256, 1, 0), (515, 515, 117, 1, 0),
                                             (640, 384, 320, 0, 1)])
def test_rank_update_rounded(h, dt, M, N, K, lower, kxn):
    g = torch.Generator().manual_seed(11 + K)
    X = torch.randn((M, K), generator=g)
    Y = X.clone() if (lower and M == N) else torch.randn((K, N) if kxn else (N, K), generator=g)
    C0 = torch.randn((M, N), generator=g) * 10
    exp, Pa = _expected(C0, X, Y, kxn, dt)
    C = _run(h, dt, lower, kxn, C0.to(DEV), X.to(DEV), Y.to(DEV)).cpu().double()
    err = (C - exp).abs()
    tol = 4e-6 * (C0.double().abs() + Pa)
    if lower:
        mask = torch.tril(torch.ones(M, N, dtype=torch.bool))
        assert bool((err[mask] <= tol[mask]).all())
        assert torch.equal(C[~mask], C0.double()[~mask])
    else:
        assert bool((err <= tol).all())


def test_rank_update_strided_views(h):
    """Operands that are views into a larger matrix (the panel of W)."""
    n, z, s = 700, 100, 130
    W = torch.randint(-3, 4, (n, n + 5), dtype=torch.float32)
    C0 = W.clone()
    c = z + s
    Wd = W.to(DEV)
    Cv = Wd[c:, c:n]
    R = Wd[c:, z:c]
    _run(h, "mix_bf16", 1, 0, Cv, R, R)
    Rh = C0[c:, z:c].double()
    exp = C0[c:, c:n].double() - Rh @ Rh.T
    got = Wd[c:, c:n].cpu().double()
    mask = torch.tril(torch.ones(n - c, n - c, dtype=torch.bool))
    assert torch.equal(got[mask], exp[mask])
    rest = Wd.cpu()
    rest[c:, c:n] = C0[c:, c:n]
    assert torch.equal(rest, C0)  # nothing outside the trailing block changed


def test_rank_update_preserves_negative_zero_above_diagonal(h):
    """Masked entries of diagonal tiles receive -0.0 (x + -0 == x for every x)."""
    M = 300
    C0 = torch.full((M, M), -0.0)
    X = torch.ones((M, 64))
    C = _run(h, "mix_bf16", 1, 0, C0.to(DEV), X.to(DEV), X.to(DEV)).cpu()
    up = torch.triu(torch.ones(M, M, dtype=torch.bool), 1)
    assert bool(torch.signbit(C[up]).all())
    assert bool((C[~up] == -64.0).all())


def test_bf16x3_is_fp32_accurate_where_bf16_is_not(h):
    """Non-representable operands: plain BF16 errs at ~2^-9 per product, the split
    only by FP32 accumulation."""
    g = torch.Generator().manual_seed(3)
    M, K = 256, 512
    X = torch.rand((M, K), generator=g) + 0.5
    C0 = torch.zeros((M, M))
    ref = -(X.double() @ X.double().T)
    errs = {}
    for dt in ("mix_bf16", "mix_bf16x3"):
        C = _run(h, dt, 0, 0, C0.clone().to(DEV), X.to(DEV), X.to(DEV)).cpu().double()
        errs[dt] = ((C - ref).abs() / ref.abs()).max().item()
    assert errs["mix_bf16"] > 1e-4
    assert errs["mix_bf16x3"] < 2e-5


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("M,N,K,kxn", [(1024, 1024, 128, 1), (1001, 777, 129, 1),
                                       (777, 1001, 64, 0), (2048, 600, 255, 0)])
def test_strassen_matches_classical_on_exact_integers(h, dt, M, N, K, kxn):
    """Every sum Strassen forms is exact for small integers, so one level must
    give the same bits as the classical update (odd sizes take the classical
    remainders)."""
    from paper_1812_02056_gb300 import binding
    g = torch.Generator().manual_seed(M + N + K)
    tt = torch.float64 if dt == "f64" else torch.float32
    X = torch.randint(-4, 5, (M, K), generator=g).to(tt)
    Y = torch.randint(-4, 5, (K, N) if kxn else (N, K), generator=g).to(tt)
    C0 = torch.randint(-1000, 1000, (M, N), generator=g).to(tt)
    exp, _ = _expected(C0, X, Y, kxn, dt)
    h.set_option(binding.GB_OPT_STRASSEN, 1)
    try:
        C = _run(h, dt, 0, kxn, C0.to(DEV), X.to(DEV), Y.to(DEV)).cpu().double()
    finally:
        h.set_option(binding.GB_OPT_STRASSEN, 0)
    assert torch.equal(C, exp)


@pytest.mark.parametrize("kind", ["chol", "lu"])
def test_factorizations_with_strassen_match_oracle(h, kind):
    import oracle
    from paper_1812_02056_gb300 import binding
    from paper_1812_02056_gb300 import inputs as I
    from tests.helpers import guarded_rel_err, lu_split
    n, s = 2600, 1100
    A = I.spd_gram(n, 3) if kind == "chol" else I.lu_diag_dominant(n, 3)
    Ad = torch.from_numpy(A).to(DEV)
    h.set_option(binding.GB_OPT_STRASSEN, 1)
    try:
        F, info = (h.chol_factor if kind == "chol" else h.lu_factor)(Ad, s, "f64")
    finally:
        h.set_option(binding.GB_OPT_STRASSEN, 0)
    assert int(info.item()) == 0
    Fg = F.cpu().numpy()
    if kind == "chol":
        Lo, _ = oracle.chol(A, s)
        assert guarded_rel_err(Fg, Lo) <= 1e-10
        assert h.backward_error(Ad, F, "f64") <= 1e-13
    else:
        Lo, Uo, _ = oracle.lu(A, s)
        L, U = lu_split(Fg)
        assert guarded_rel_err(L, Lo) <= 1e-10 and guarded_rel_err(U, Uo) <= 1e-10
        assert h.backward_error(Ad, F, "f64", lu=True) <= 1e-13
