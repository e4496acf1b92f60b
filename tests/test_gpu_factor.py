"""Parity of the CUDA factorizations with the FP64 oracle (Algorithms 1, 2).

Tolerances:
* FP64: elementwise guarded relative error <= 1e-10 against the oracle's
  factor, backward error <= 1e-13 (the stated FP64 bar);
* FP32: guarded relative error <= 2e-4 with the guard at 1e-2 max|L| (an
  entry's error is absolute, ~ u32 sqrt(n) times its row's norm, so tiny
  entries are compared on the scale of the largest ones), and backward
  error <= 2e-6 (single precision unit roundoff 6e-8 times the growth of
  the n <= 512 sums);
* exact integer cases (Pascal, integer factors) must agree bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests.helpers import guarded_rel_err, lu_split

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


def _chol(h, A, s, dtype="f64"):
    tt = torch.float32 if dtype == "f32" else torch.float64
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(DEV, tt)
    L, info = h.chol_factor(Ad, s, dtype)
    torch.cuda.synchronize()
    return L.double().cpu().numpy(), int(info.item())


def _lu(h, A, s, dtype="f64"):
    tt = torch.float32 if dtype == "f32" else torch.float64
    Ad = torch.from_numpy(np.ascontiguousarray(A)).to(DEV, tt)
    LU, info = h.lu_factor(Ad, s, dtype)
    torch.cuda.synchronize()
    return LU.double().cpu().numpy(), int(info.item())


SIZES = [1, 2, 3, 16, 31, 33, 64, 65, 100, 129, 200]
STEPS = [1, 2, 7, 32, 64, 65, 117, "n", "n+5"]


def _step(s, n):
    return n if s == "n" else (n + 5 if s == "n+5" else s)


# ------------------------------------------------------------------ Cholesky
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("s", STEPS)
def test_chol_f64_matches_oracle(h, n, s):
    s = _step(s, n)
    A = I.spd_gram(n, I.seed_for(I.W_SMALL, n))
    L, info = _chol(h, A, s)
    Lo, info_o = oracle.chol(A, s)
    assert info == info_o == 0
    assert np.all(np.triu(L, 1) == 0.0)
    assert guarded_rel_err(L, Lo) <= 1e-10
    assert oracle.chol_backward_error(A, L) <= 1e-13


@pytest.mark.parametrize("n", [16, 26])
@pytest.mark.parametrize("s", [1, 3, 5, 16, 40])
def test_chol_pascal_exact_f64(h, n, s):
    L, info = _chol(h, I.pascal_sym(n), s)
    assert info == 0 and np.array_equal(L, I.pascal_lower(n))


@pytest.mark.parametrize("s", [1, 4, 14])
def test_chol_pascal_exact_f32(h, s):
    L, info = _chol(h, I.pascal_sym(14), s, "f32")
    assert info == 0 and np.array_equal(L, I.pascal_lower(14))


@pytest.mark.parametrize("s", [1, 5, 64, 100])
def test_chol_integer_factor_exact(h, s):
    n = 150
    L0 = I.unit_lower_integer(n, 3)
    L, info = _chol(h, L0 @ L0.T, s)
    assert info == 0 and np.array_equal(L, L0)


@pytest.mark.parametrize("inner", [1, 8, 17, 64])
def test_chol_inner_step(h, inner):
    from paper_1812_02056_gb300 import binding
    n, s = 300, 117
    A = I.spd_gram(n, 42)
    Lo, _ = oracle.chol(A, s)
    h.set_option(binding.GB_OPT_INNER_STEP, inner)
    try:
        L, info = _chol(h, A, s)
    finally:
        h.set_option(binding.GB_OPT_INNER_STEP, 64)
    assert info == 0 and guarded_rel_err(L, Lo) <= 1e-10


@pytest.mark.parametrize("n,s", [(33, 7), (200, 32), (512, 32), (300, 117)])
def test_chol_f32_matches_oracle(h, n, s):
    A = I.spd_gram(n, 7 + n)
    A32 = A.astype(np.float32).astype(np.float64)
    L, info = _chol(h, A32, s, "f32")
    Lo, _ = oracle.chol(A32, s)
    assert info == 0
    assert guarded_rel_err(L, Lo, floor=1e-2) <= 2e-4
    assert oracle.chol_backward_error(A32, L) <= 2e-6


def test_chol_config_small(h):
    """FP64, n = 512, s = 32, A = G G^T + 512 I."""
    n, s = 512, 32
    A = I.spd_gram(n, I.seed_for(I.W_SMALL))
    L, info = _chol(h, A, s)
    Lo, _ = oracle.chol(A, s)
    assert info == 0 and guarded_rel_err(L, Lo) <= 1e-10
    be_o = oracle.chol_backward_error(A, L)
    Ad = torch.from_numpy(A).to(DEV)
    be_g = h.backward_error(Ad, torch.from_numpy(L).to(DEV), "f64")
    # at ~1e-16 the FP64 residual's own rounding is of the same size as the
    # residual: agreement is absolute there
    assert be_o <= 1e-13 and abs(be_g - be_o) <= 2e-16
    # on a perturbed factor the FP64 device residual matches the long-double one
    Lp = L * (1.0 + 1e-8 * np.cos(np.arange(n))[None, :])
    be_o = oracle.chol_backward_error(A, Lp)
    be_g = h.backward_error(Ad, torch.from_numpy(Lp).to(DEV), "f64")
    assert abs(be_g - be_o) <= 1e-3 * be_o


def test_chol_in_place_and_padded_ld(h):
    n, s = 150, 20
    A = I.spd_gram(n, 11)
    Lo, _ = oracle.chol(A, s)
    big = torch.zeros((n, n + 9), dtype=torch.float64, device=DEV)
    big[:, :n] = torch.from_numpy(A).to(DEV)
    view = big[:, :n]
    from paper_1812_02056_gb300 import binding
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    st = h.gb_chol_factor(n, s, binding.GB_F64, view, n + 9, view, n + 9, info)
    assert st == 0
    torch.cuda.synchronize()
    L = view.cpu().numpy()
    assert int(info.item()) == 0 and guarded_rel_err(L, Lo) <= 1e-10
    assert np.all(big[:, n:].cpu().numpy() == 0.0)  # padding untouched


def test_chol_host_buffers_match_device(h):
    from paper_1812_02056_gb300 import binding
    n, s = 257, 64
    A = I.spd_gram(n, 13)
    L = np.zeros((n, n))
    info = np.zeros(1, dtype=np.int32)
    st = h.gb_chol_factor(n, s, binding.GB_F64, A, n, L, n, info)
    assert st == 0 and info[0] == 0
    Ld, _ = _chol(h, A, s)
    assert np.array_equal(L, Ld)


@pytest.mark.parametrize("dtype", ["f64", "f32", "mix_bf16", "mix_bf16x3"])
@pytest.mark.parametrize("n,s", [(257, 64), (300, 200), (1000, 256), (1000, 1000), (2000, 128)])
def test_chol_host_buffers_streamed_by_column_blocks(h, dtype, n, s):
    """Host buffers: A goes in by column slabs (lower triangle only) while the
    factorization starts, with the first trailing update in strips that wait
    for their slab, and the finished block columns go out while it goes on.
    The host L (padded pitch, filled with NaN) must hold the device-buffer
    factor bit for bit, zeros above the diagonal, and untouched padding."""
    from paper_1812_02056_gb300 import binding
    dt = binding.DTYPES[dtype]
    A = I.spd_gram(n, 17 + n)
    Ain = A.astype(np.float32) if dtype == "f32" else A
    fdt = np.float64 if dtype == "f64" else np.float32
    ldl = n + 3
    Lh = np.full((n, ldl), np.nan, dtype=fdt)
    info = np.zeros(1, dtype=np.int32)
    st = h.gb_chol_factor(n, s, dt, Ain, n, Lh, ldl, info)
    assert st == 0 and info[0] == 0
    Ad = torch.from_numpy(Ain).to(DEV)
    Ld = torch.empty((n, n), dtype=torch.float64 if dtype == "f64" else torch.float32, device=DEV)
    infod = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert h.gb_chol_factor(n, s, dt, Ad, n, Ld, n, infod) == 0
    torch.cuda.synchronize()
    assert np.array_equal(Lh[:, :n], Ld.cpu().numpy())
    assert np.all(np.triu(Lh[:, :n], 1) == 0.0)
    assert np.all(np.isnan(Lh[:, n:]))
    # host input, device output (NaN in A's upper triangle is never read)
    Au = Ain.copy()
    Au[np.triu_indices(n, 1)] = np.nan
    L2 = torch.full((n, n), float("nan"), dtype=Ld.dtype, device=DEV)
    assert h.gb_chol_factor(n, s, dt, Au, n, L2, n, infod) == 0
    torch.cuda.synchronize()
    assert int(infod.item()) == 0
    assert torch.equal(L2, Ld)


def test_chol_breakdown_reports_column(h):
    n = 100
    A = I.spd_gram(n, 1)
    A[37, 37] = -1e7
    for s in [1, 16, 64, 100]:
        _, info = _chol(h, A, s)
        assert info == 38
    _, info = _chol(h, np.array([[1.0, 2.0], [2.0, 1.0]]), 1)
    assert info == 2
    B = I.spd_gram(20, 2)
    B[5, 3] = B[3, 5] = np.nan
    _, info = _chol(h, B, 4)
    assert info > 0


@pytest.mark.parametrize("dtype", ["f32", "mix_bf16", "mix_bf16x3"])
def test_chol_breakdown_reports_column_fp32_working_matrix(h, dtype):
    """The FP32 and mixed paths (one warp finishes each 16-column chunk of
    the diagonal block) report the first non-positive pivot, inside and
    across chunks and inner blocks, and a NaN anywhere."""
    n = 300
    for k in (0, 15, 16, 137, 299):
        A = I.spd_gram(n, 1)
        A[k, k] = -1e7
        for s in [16, 64, 100, 300]:
            _, info = _chol(h, A, s, dtype)
            assert info == k + 1, (k, s)
    B = I.spd_gram(40, 2)
    B[25, 3] = B[3, 25] = np.nan
    _, info = _chol(h, B, 8, dtype)
    assert info > 0


def test_chol_empty(h):
    from paper_1812_02056_gb300 import binding
    info = np.ones(1, dtype=np.int32)
    assert h.gb_chol_factor(0, 4, binding.GB_F64, None, 1, None, 1, info) == 0
    assert info[0] == 0


def test_argument_errors(h):
    from paper_1812_02056_gb300 import binding
    A = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    info = torch.zeros(1, dtype=torch.int32, device=DEV)
    assert h.gb_chol_factor(-1, 2, 0, A, 4, A, 4, info) == -2
    assert h.gb_chol_factor(4, -2, 0, A, 4, A, 4, info) == -3
    assert h.gb_chol_factor(4, 2, 9, A, 4, A, 4, info) == -4
    assert h.gb_chol_factor(4, 2, 0, A, 3, A, 4, info) == -6
    assert h.gb_chol_factor(4, 2, 0, A, 4, A, 4, None) == -9
    # mixed in place is refused (FP64 input, FP32 factor)
    assert h.gb_chol_factor(4, 2, binding.GB_MIX_BF16, A, 4, A, 4, info) == -7


# ------------------------------------------------------------------------ LU
@pytest.mark.parametrize("n", [1, 2, 5, 33, 64, 65, 130, 200])
@pytest.mark.parametrize("s", [1, 3, 32, 64, 65, 117, "n", "n+5"])
def test_lu_f64_matches_oracle(h, n, s):
    s = _step(s, n)
    A = I.lu_diag_dominant(n, I.seed_for(I.W_N8192, n))
    LU, info = _lu(h, A, s)
    Lo, Uo, info_o = oracle.lu(A, s)
    assert info == info_o == 0
    L, U = lu_split(LU)
    assert guarded_rel_err(L, Lo) <= 1e-10
    assert guarded_rel_err(U, Uo) <= 1e-10
    assert oracle.lu_backward_error(A, L, U) <= 1e-13


@pytest.mark.parametrize("s", [1, 4, 16, 30])
def test_lu_pascal_exact(h, s):
    LU, info = _lu(h, I.pascal_sym(16), s)
    L, U = lu_split(LU)
    P = I.pascal_lower(16)
    assert info == 0 and np.array_equal(L, P) and np.array_equal(U, P.T)


@pytest.mark.parametrize("s", [1, 7, 64, 90])
def test_lu_integer_factors_exact(h, s):
    n = 120
    L0 = I.unit_lower_integer(n, 5)
    U0 = I.unit_lower_integer(n, 6).T
    LU, info = _lu(h, L0 @ U0, s)
    L, U = lu_split(LU)
    assert info == 0 and np.array_equal(L, L0) and np.array_equal(U, U0)


def test_lu_f32(h):
    n, s = 300, 64
    A = I.lu_diag_dominant(n, 3).astype(np.float32).astype(np.float64)
    LU, info = _lu(h, A, s, "f32")
    Lo, Uo, _ = oracle.lu(A, s)
    L, U = lu_split(LU)
    assert info == 0
    assert guarded_rel_err(L, Lo, floor=1e-2) <= 2e-4
    assert guarded_rel_err(U, Uo, floor=1e-2) <= 2e-4
    assert oracle.lu_backward_error(A, L, U) <= 2e-6


def test_lu_breakdown(h):
    A = I.lu_diag_dominant(50, 4)
    A[:13, :13] = 1.0  # leading minor of order 2 vanishes
    _, info = _lu(h, A, 8)
    assert info == 2


@pytest.mark.parametrize("inner", [1, 13, 64])
def test_lu_inner_step(h, inner):
    from paper_1812_02056_gb300 import binding
    n, s = 260, 117
    A = I.lu_diag_dominant(n, 9)
    Lo, Uo, _ = oracle.lu(A, s)
    h.set_option(binding.GB_OPT_INNER_STEP, inner)
    try:
        LU, info = _lu(h, A, s)
    finally:
        h.set_option(binding.GB_OPT_INNER_STEP, 64)
    L, U = lu_split(LU)
    assert info == 0 and guarded_rel_err(L, Lo) <= 1e-10 and guarded_rel_err(U, Uo) <= 1e-10


@pytest.mark.parametrize("rec", [0, 1])
@pytest.mark.parametrize("n,s", [(1000, 512), (777, 300), (2048, 1024)])
def test_inner_halves_and_flat_match_oracle(h, rec, n, s):
    """GB_OPT_INNER_RECURSIVE: an s-block's columns finished in halves (the
    right half receiving the whole left half in one product) or inner block
    by inner block: FP64 against the oracle at the suite's tolerance, and the
    mixed factor of an integer L0 L0^T exactly L0 either way."""
    from paper_1812_02056_gb300 import binding
    prev = h.get_option(binding.GB_OPT_INNER_RECURSIVE)
    assert prev == 2  # the default
    h.set_option(binding.GB_OPT_INNER_RECURSIVE, rec)
    try:
        A = I.spd_gram(n, 500 + n)
        L, info = _chol(h, A, s)
        assert info == 0
        Lo, _ = oracle.chol(A, s)
        assert guarded_rel_err(L, Lo) <= 1e-10
        L0 = I.unit_lower_integer(n, 600 + n, -1, 1)
        for dt in ("mix_bf16", "mix_bf16x3"):
            Lm, info = _chol(h, L0 @ L0.T, s, dt)
            assert info == 0 and np.array_equal(Lm, L0)
    finally:
        h.set_option(binding.GB_OPT_INNER_RECURSIVE, prev)
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_INNER_RECURSIVE, 3) == -3


@pytest.mark.parametrize("dtype", ["f64", "f32", "mix_bf16", "mix_bf16x3"])
@pytest.mark.parametrize("n,s", [(2000, 512), (1500, 256), (700, 1024)])
def test_inner_lookahead_same_bits(h, dtype, n, s):
    """GB_OPT_INNER_LOOKAHEAD splits each product inside an s-block into the
    next inner block's columns and the rest of the range, on two streams:
    every element receives the same sums in the same order, so the factor is
    the same bits with and without it (and matches the oracle)."""
    from paper_1812_02056_gb300 import binding
    A = I.spd_gram(n, 900 + n)
    assert h.get_option(binding.GB_OPT_INNER_LOOKAHEAD) == 2  # the default: FP64 only
    try:
        h.set_option(binding.GB_OPT_INNER_LOOKAHEAD, 0)
        L0, info0 = _chol(h, A, s, dtype)
        h.set_option(binding.GB_OPT_INNER_LOOKAHEAD, 1)
        L1, info1 = _chol(h, A, s, dtype)
    finally:
        h.set_option(binding.GB_OPT_INNER_LOOKAHEAD, 2)
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_INNER_LOOKAHEAD, 3) == -3
    assert info0 == 0 and info1 == 0
    assert np.array_equal(L0, L1)
    if dtype == "f64":
        Lo, _ = oracle.chol(A, s)
        assert guarded_rel_err(L1, Lo) <= 1e-10


@pytest.mark.parametrize("dtype", ["f64", "f32", "mix_bf16x3"])
@pytest.mark.parametrize("n,s", [(2000, 512), (1500, 256), (1100, 128)])
def test_early_rest_same_bits(h, dtype, n, s):
    """GB_OPT_EARLY_REST starts the rest of each delayed update (the columns
    after the next s-block) before the next s-block's own update: the two
    write disjoint columns and read only finished ones, so the factor is the
    same bits either way (and matches the oracle)."""
    from paper_1812_02056_gb300 import binding
    A = I.spd_gram(n, 1300 + n)
    assert h.get_option(binding.GB_OPT_EARLY_REST) == 2  # the default: FP64 only
    try:
        h.set_option(binding.GB_OPT_EARLY_REST, 0)
        L0, info0 = _chol(h, A, s, dtype)
        h.set_option(binding.GB_OPT_EARLY_REST, 1)
        L1, info1 = _chol(h, A, s, dtype)
    finally:
        h.set_option(binding.GB_OPT_EARLY_REST, 2)
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_EARLY_REST, 3) == -3
    assert info0 == 0 and info1 == 0
    assert np.array_equal(L0, L1)
    if dtype == "f64":
        Lo, _ = oracle.chol(A, s)
        assert guarded_rel_err(L1, Lo) <= 1e-10
