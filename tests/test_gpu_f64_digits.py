"""The FP64 delayed update of Algorithm 1 to FP64 accuracy from exact digit
products on the tensor cores (GB_OPT_F64_UPDATE = 1), against exact and
oracle references.

* Integer X, Y, C whose products and sums are exact in FP64: the update
  C -= X Y^T (lower) is exact, bit for bit, for X = Y (one set of digits)
  and X != Y, with K up to 1500 (K taken in pieces of at most 1024).
* Random X with a spread of magnitudes against the correctly rounded
  result (Veltkamp splitting, math.fsum): the error is below
  2^-48 2^(e_i + e_j), 2^e_i the power of two that scales row i.  A dropped
  scale or a wrong digit plane errs by 2^-44 or more of that.
* gb_chol_factor with the option: the factor within 1e-10 of the oracle's
  (elementwise, guarded), backward error <= 1e-13, the same bits with and
  without look-ahead, breakdown reported as usual; at the benchmark's
  n = 8192, s = 256 against the oracle's whole factor.
* Algorithm 2's general update (every element, R_U stored K x N) exact on
  integers, and gb_lu_factor with the option against the oracle's L and U
  (1e-10, backward error <= 1e-13) and exact on integer factors.
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests.helpers import exact_dot_minus, guarded_rel_err, pow2_scale

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


class _digits:
    """GB_OPT_F64_UPDATE = v inside the block."""

    def __init__(self, h, v=1):
        self.h, self.v = h, v

    def __enter__(self):
        from paper_1812_02056_gb300 import binding
        self.prev = self.h.get_option(binding.GB_OPT_F64_UPDATE)
        self.h.set_option(binding.GB_OPT_F64_UPDATE, self.v)

    def __exit__(self, *a):
        from paper_1812_02056_gb300 import binding
        self.h.set_option(binding.GB_OPT_F64_UPDATE, self.prev)


def _rank_update(h, C, X, Y, N=None):
    """C -= X Y^T (lower); Y None: Y is X's first N rows (the same buffer)."""
    from paper_1812_02056_gb300 import binding
    M, K = X.shape
    N = Y.shape[0] if Y is not None else (M if N is None else N)
    Cd = _t(C)
    Xd = _t(X)
    Yd = Xd if Y is None else _t(Y)
    st = h.gb_rank_update(binding.GB_F64, 1, 0, M, N, K, Cd, N, Xd, K, Yd, K)
    assert st == 0, binding.status_string(st)
    torch.cuda.synchronize()
    return Cd.cpu().numpy()


def test_option_default_and_range(h):
    from paper_1812_02056_gb300 import binding
    assert h.get_option(binding.GB_OPT_F64_UPDATE) == 0
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_F64_UPDATE, 2) == -3


@pytest.mark.parametrize("M,N,K,same", [(300, 300, 1, True), (1000, 1000, 37, True),
                                        (2100, 777, 256, False), (1300, 1300, 1500, True),
                                        (515, 300, 1100, False)])
def test_integer_update_is_exact(h, M, N, K, same):
    rng = np.random.default_rng(M + N + K)
    X = rng.integers(-1000, 1001, (M, K))
    Y = X[:N] if same else rng.integers(-1000, 1001, (N, K))
    C = rng.integers(-10 ** 9, 10 ** 9, (M, N))
    ref = C - X @ Y.T  # int64: exact
    mask = np.tril(np.ones((M, N), dtype=bool))
    with _digits(h):
        got = _rank_update(h, C.astype(np.float64), X.astype(np.float64),
                           None if same else Y.astype(np.float64), N)
    assert np.array_equal(got[mask], ref[mask].astype(np.float64))
    assert np.array_equal(got[~mask], C[~mask].astype(np.float64))  # above the diagonal: untouched


@pytest.mark.parametrize("M,K", [(700, 256), (1500, 64)])
def test_update_against_correctly_rounded(h, M, K):
    rng = np.random.default_rng(M * K)
    X = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-2, 2, (M, 1))
    X *= 10.0 ** rng.uniform(-1, 1, (1, K))
    C = rng.standard_normal((M, M))
    with _digits(h):
        got = _rank_update(h, C, X, None)
    with _digits(h, 0):
        fma = _rank_update(h, C, X, None)
    worst = worst_f = 0.0
    u = 2.0 ** -53
    for i in sorted({0, 1, M // 2, M - 1, *rng.integers(0, M, 12).tolist()}):
        for j in sorted({0, i, *rng.integers(0, i + 1, 8).tolist()}):
            ref = exact_dot_minus(C[i, j], X[i], X[j])
            # the product's scale, plus the rounding of the result itself
            scale = pow2_scale(X[i]) * pow2_scale(X[j])
            worst = max(worst, max(abs(got[i, j] - ref) - 2 * u * abs(ref), 0.0) / scale)
            worst_f = max(worst_f, max(abs(fma[i, j] - ref) - 2 * u * abs(ref), 0.0) / scale)
    assert worst <= 2.0 ** -48, (worst, worst_f)
    assert worst_f <= K * 2.0 ** -52


@pytest.mark.parametrize("n,s", [(200, 32), (1000, 256), (2600, 512), (3001, 300)])
def test_chol_f64_digits_matches_oracle(h, n, s):
    A = I.spd_gram(n, 400 + n)
    with _digits(h):
        L, info = h.chol_factor(_t(A), s, "f64")
    assert int(info.item()) == 0
    Lg = L.cpu().numpy()
    assert np.all(np.triu(Lg, 1) == 0.0)
    Lo, _ = oracle.chol(A, s)
    assert guarded_rel_err(Lg, Lo) <= 1e-10
    assert oracle.chol_backward_error(A, Lg) <= 1e-13


def test_chol_f64_digits_same_bits_with_and_without_lookahead(h):
    from paper_1812_02056_gb300 import binding
    n, s = 2600, 256
    A = _t(I.spd_gram(n, 77))
    with _digits(h):
        L1, _ = h.chol_factor(A, s, "f64")
        h.set_option(binding.GB_OPT_LOOKAHEAD, 0)
        try:
            L0, _ = h.chol_factor(A, s, "f64")
        finally:
            h.set_option(binding.GB_OPT_LOOKAHEAD, 1)
    assert torch.equal(torch.tril(L0), torch.tril(L1))


def test_chol_f64_digits_breakdown(h):
    n = 700
    A = I.spd_gram(n, 9)
    A[450, 450] = -1.0  # the leading 450 x 450 block stays SPD
    with _digits(h):
        _, info = h.chol_factor(_t(A), 128, "f64")
    _, info_o = oracle.chol(A, 128)
    assert int(info.item()) == info_o == 451


def test_chol_f64_digits_n8192_full_oracle(h):
    A = I.spd_gram(8192, I.seed_for(I.W_N8192, 0), device=DEV)  # bench.py's input
    with _digits(h):
        L, info = h.chol_factor(A, 256, "f64")
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert h.backward_error(A, L, "f64") <= 1e-13
    Lo, info_o = oracle.chol(A.cpu().numpy(), 256)
    assert info_o == 0
    assert guarded_rel_err(L.cpu().numpy(), Lo) <= 1e-10


def _general_update(h, C, X, Y, y_kxn):
    """C -= X op(Y) over every element (gb_rank_update with lower = 0)."""
    from paper_1812_02056_gb300 import binding
    M, K = X.shape
    N = Y.shape[1] if y_kxn else Y.shape[0]
    Cd, Xd, Yd = _t(C), _t(X), _t(Y)
    st = h.gb_rank_update(binding.GB_F64, 0, int(y_kxn), M, N, K, Cd, N, Xd, K, Yd,
                          N if y_kxn else K)
    assert st == 0, binding.status_string(st)
    torch.cuda.synchronize()
    return Cd.cpu().numpy()


@pytest.mark.parametrize("M,N,K,y_kxn", [(700, 1300, 300, True), (2100, 500, 1100, True),
                                         (640, 640, 64, False), (300, 1000, 17, True)])
def test_general_integer_update_is_exact(h, M, N, K, y_kxn):
    """Algorithm 2's update (every element; R_U stored K x N and cut into
    digits by columns), and the N x K form, exact on integers."""
    rng = np.random.default_rng(M * 7 + N + K)
    X = rng.integers(-1000, 1001, (M, K))
    Y = rng.integers(-1000, 1001, (K, N) if y_kxn else (N, K))
    C = rng.integers(-10 ** 9, 10 ** 9, (M, N))
    ref = C - X @ (Y if y_kxn else Y.T)
    with _digits(h):
        got = _general_update(h, C.astype(np.float64), X.astype(np.float64),
                              Y.astype(np.float64), y_kxn)
    assert np.array_equal(got, ref.astype(np.float64))


@pytest.mark.parametrize("n,s", [(300, 32), (1000, 256), (2600, 512), (3001, 300)])
def test_lu_f64_digits_matches_oracle(h, n, s):
    from tests.helpers import lu_split
    A = I.lu_diag_dominant(n, 500 + n)
    with _digits(h):
        LU, info = h.lu_factor(_t(A), s, "f64")
    assert int(info.item()) == 0
    L, U = lu_split(LU.cpu().numpy())
    Lo, Uo, info_o = oracle.lu(A, s)
    assert info_o == 0
    assert guarded_rel_err(L, Lo) <= 1e-10
    assert guarded_rel_err(U, Uo) <= 1e-10
    assert oracle.lu_backward_error(A, L, U) <= 1e-13


@pytest.mark.parametrize("s", [7, 64])
def test_lu_f64_digits_integer_factors_exact(h, s):
    from tests.helpers import lu_split
    n = 120
    L0 = I.unit_lower_integer(n, 5)
    U0 = I.unit_lower_integer(n, 6).T
    with _digits(h):
        LU, info = h.lu_factor(_t(L0 @ U0), s, "f64")
    L, U = lu_split(LU.cpu().numpy())
    assert int(info.item()) == 0 and np.array_equal(L, L0) and np.array_equal(U, U0)
