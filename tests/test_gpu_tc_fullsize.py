"""Tensor-core parity at full size.

At n = 8192 every CTA (or CTA pair) of the persistent tensor-core update
processes several output tiles, so its accumulator double buffer is reused
and its shared-memory ring wraps around many times; smaller cases give each
cluster at most one tile.

* The update alone (Sec. 2, Algorithm 1: A[c.., c..] -= R R^T): small
  integer operands make every product and partial sum exact in BF16/FP16
  operands and FP32 accumulators, so C - tril(X X^T) must come out bit for
  bit, for every mixed dtype, K in {1024, 2048} and both the one-CTA and the
  CTA-pair kernel.  The expected matrix is computed on the host.
* The whole mixed factorization: A = L0 L0^T with L0 unit lower and entries
  in {-1, 0, 1} keeps every intermediate value a small integer, so the
  factor must be L0 bit for bit, right- and left-looking, s in {512, 1024}.
* Rounded: the BF16x3 and FP32 factors at n = 4096 against the FP64 oracle,
  entry by entry, in units of their rounding model (tests.helpers.
  row_scaled_err: u sqrt(j + 1) times the row's typical entry, with u the
  FP32 unit roundoff 2^-24; BF16x3 operands carry 24 bits, so its products
  round like FP32).
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests.helpers import row_scaled_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
N = 8192
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


@pytest.fixture(scope="module", params=[1024, 2048])
def update_case(request):
    """X (N x K) and C0 (N x N) of small integers, and C0 - tril(X X^T)
    computed on the host in FP64 (exact: every value is an integer below 2^24)."""
    K = request.param
    g = I.rng(9000 + K)
    X = g.integers(-4, 5, size=(N, K)).astype(np.float32)
    C0 = g.integers(-1000, 1001, size=(N, N)).astype(np.float32)
    X64 = X.astype(np.float64)
    exp = C0.astype(np.float64) - np.tril(X64 @ X64.T)
    assert np.abs(exp).max() < 2 ** 24
    return K, torch.from_numpy(X).to(DEV), torch.from_numpy(C0).to(DEV), \
        torch.from_numpy(exp.astype(np.float32)).to(DEV)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
def test_rank_update_exact_integers_n8192(h, update_case, dt, mode):
    from paper_1812_02056_gb300 import binding
    K, X, C0, exp = update_case
    C = C0.clone()
    prev = h.get_option(binding.GB_OPT_TC_UPDATE)
    h.set_option(binding.GB_OPT_TC_UPDATE, mode)
    try:
        binding.check(h.gb_rank_update(binding.DTYPES[dt], 1, 0, N, N, K, C, N, X, K, X, K),
                      "gb_rank_update")
        torch.cuda.synchronize()
    finally:
        h.set_option(binding.GB_OPT_TC_UPDATE, prev)
    # lower triangle updated exactly, strict upper part untouched
    bad = int((C != exp).sum().item())
    assert bad == 0, f"{bad} entries differ"


@pytest.fixture(scope="module")
def integer_spd():
    L0 = I.unit_lower_integer(N, 9100, -1, 1)
    L0d = torch.from_numpy(L0).to(DEV)
    A = L0d @ L0d.T  # exact: integers below 2^24
    assert float(A.abs().max().item()) < 2 ** 24
    return A, L0d


@pytest.mark.parametrize("left", [False, True])
@pytest.mark.parametrize("s", [512, 1024])
@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
def test_mixed_chol_integer_factor_n8192(h, integer_spd, dt, s, left):
    from paper_1812_02056_gb300 import binding
    if left and dt == "mix_bf16x3":
        pytest.skip("left-looking accumulation keeps one 16-bit plane (BF16, FP16)")
    A, L0d = integer_spd
    h.set_option(binding.GB_OPT_LEFT_LOOKING, 1 if left else 0)
    try:
        L, info = h.chol_factor(A, s, dt)
        torch.cuda.synchronize()
    finally:
        h.set_option(binding.GB_OPT_LEFT_LOOKING, 0)
    assert int(info.item()) == 0
    bad = int((L.double() != L0d).sum().item())
    assert bad == 0, f"{bad} entries differ from L0"


# measured maxima of row_scaled_err are a few units (random-sign rounding);
# the bounds leave a margin of about 4x and stay far below the 1/u that a
# dropped or wrong term produces
ROW_SCALED_BOUND = {"gram": 16.0, "logspaced": 16.0 * 100.0}


@pytest.mark.parametrize("matrix", ["gram", "logspaced"])
@pytest.mark.parametrize("dt,s", [("mix_bf16x3", 512), ("f32", 256)])
def test_factor_n4096_vs_oracle_elementwise(h, dt, s, matrix):
    """A = G G^T + n I (cond ~ 5) and the mixed-precision workload's
    Q diag(sigma) Q^T (cond 1e4, whose forward error may grow by up to
    cond^(1/2) = 100)."""
    n = 4096
    if matrix == "gram":
        A = I.spd_gram(n, 9200)
    else:
        A = I.spd_logspaced(n, 9201, cond=1e4)
    Ain = torch.from_numpy(A).to(DEV)
    if dt == "f32":
        Ain = Ain.float()
        A = Ain.double().cpu().numpy()  # the oracle factors the FP32 input exactly
    L, info = h.chol_factor(Ain, s, dt)
    assert int(info.item()) == 0
    Lg = L.double().cpu().numpy()
    Lo, info_o = oracle.chol(A, s)
    assert info_o == 0
    e = row_scaled_err(Lg, Lo, U32)
    assert e <= ROW_SCALED_BOUND[matrix], f"row-scaled error {e:.2f}"
    be = oracle.chol_backward_error(A, Lg)
    assert be <= 8 * np.sqrt(n) * U32, f"backward error {be:.3e}"
