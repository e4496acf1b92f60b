"""Algorithm 3 (fast QR, block Gram-Schmidt) on the GPU against the oracle.

The QR of a nonsingular matrix with diag(R) > 0 is unique, so the GPU's Q
and R are compared with the oracle's element by element.  The GPU adds its
dot products in a different order (cluster-wide tree sums) and, for s above
its inner step, projects the columns inside an s-block in inner blocks, so
the comparison allows Gram-Schmidt's rounding: 10 n u cond(A) (u the unit
roundoff of the arithmetic).  Exact cases: A = P R0 (permutation times an
integer upper triangle) gives Q = P and R = R0 exactly in any summation
order; rank deficiency is reported at the first zero column.
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


def perm_upper(n, seed, zero_diag_at=None):
    g = I.rng(seed)
    perm = g.permutation(n)
    P = np.zeros((n, n))
    P[perm, np.arange(n)] = 1.0
    R0 = np.triu(g.integers(-5, 6, size=(n, n)).astype(np.float64), 1)
    R0[np.diag_indices(n)] = g.integers(1, 9, size=n).astype(np.float64)
    if zero_diag_at is not None:
        R0[zero_diag_at, zero_diag_at] = 0.0
    return P @ R0, P, R0


def well_conditioned(n, seed):
    return I.gaussian(n, n, seed) + np.sqrt(n) * 2.0 * np.eye(n)


@pytest.mark.parametrize("n,s", [(1, 4), (7, 3), (64, 16), (100, 32), (300, 64), (513, 100),
                                 (1000, 256), (1200, 1200)])
def test_qr_fp64_matches_oracle(h, n, s):
    A = well_conditioned(n, 10 + n)
    Qd, Rd, info = h.qr_factor(torch.from_numpy(A).to(DEV), s, "f64")
    assert int(info.item()) == 0
    Q, R = Qd.cpu().numpy(), Rd.cpu().numpy()
    Qo, Ro, io = oracle.qr(A, s)
    assert io == 0
    tol = 10 * n * 2.0 ** -53 * np.linalg.cond(A)
    assert np.abs(Q - Qo).max() <= tol
    assert np.abs(R - Ro).max() <= tol * np.abs(Ro).max()
    assert np.array_equal(np.tril(R, -1), np.zeros((n, n)))
    assert oracle.qr_backward_error(A, Q, R) <= 1e-15 * max(n, 10)
    assert oracle.orthogonality(Q) <= 1e-15 * max(n, 10) * np.linalg.cond(A)


@pytest.mark.parametrize("n,s", [(64, 16), (500, 128)])
def test_qr_fp32_matches_oracle(h, n, s):
    A = well_conditioned(n, 20 + n).astype(np.float32)
    Qd, Rd, info = h.qr_factor(torch.from_numpy(A).to(DEV), s, "f32")
    assert int(info.item()) == 0
    Q, R = Qd.double().cpu().numpy(), Rd.double().cpu().numpy()
    Qo, Ro, _ = oracle.qr(A.astype(np.float64), s)
    tol = 10 * n * 2.0 ** -24 * np.linalg.cond(A.astype(np.float64))
    assert np.abs(Q - Qo).max() <= tol
    assert np.abs(R - Ro).max() <= tol * np.abs(Ro).max()
    assert oracle.qr_backward_error(A.astype(np.float64), Q, R) <= 1e-6 * max(n, 10) / 10


@pytest.mark.parametrize("n,s", [(5, 2), (40, 7), (200, 32), (333, 333)])
def test_qr_permutation_exact(h, n, s):
    A, P, R0 = perm_upper(n, 3 * n + s)
    Qd, Rd, info = h.qr_factor(torch.from_numpy(A).to(DEV), s, "f64")
    assert int(info.item()) == 0
    assert np.array_equal(Qd.cpu().numpy(), P)
    assert np.array_equal(Rd.cpu().numpy(), R0)


@pytest.mark.parametrize("c,s", [(0, 4), (37, 16), (99, 32)])
def test_qr_breakdown_column(h, c, s):
    A, _, _ = perm_upper(100, 50 + c, zero_diag_at=c)
    _, _, info = h.qr_factor(torch.from_numpy(A).to(DEV), s, "f64")
    assert int(info.item()) == c + 1


def test_qr_inner_step_equals_oracle_step(h):
    """With the inner step >= s the GPU runs exactly Algorithm 3's blocking;
    only the summation order differs from the oracle."""
    from paper_1812_02056_gb300 import binding
    n, s = 400, 16
    A = well_conditioned(n, 77)
    Qd, Rd, _ = h.qr_factor(torch.from_numpy(A).to(DEV), s, "f64")
    Qo, Ro, _ = oracle.qr(A, s)
    assert np.abs(Qd.cpu().numpy() - Qo).max() <= 1e-13
    assert h.get_option(binding.GB_OPT_QR_INNER_STEP) == 16
    h.set_option(binding.GB_OPT_QR_INNER_STEP, 4)
    try:
        Q4, R4, _ = h.qr_factor(torch.from_numpy(A).to(DEV), s, "f64")
    finally:
        h.set_option(binding.GB_OPT_QR_INNER_STEP, 16)
    assert np.abs(Q4.cpu().numpy() - Qo).max() <= 1e-13
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_QR_INNER_STEP, 0) == -3


def test_qr_host_buffers_and_rejections(h):
    from paper_1812_02056_gb300 import binding
    n = 50
    A = well_conditioned(n, 5)
    Q = np.zeros((n, n))
    R = np.zeros((n, n))
    info = np.zeros(1, dtype=np.int32)
    binding.check(h.gb_qr_factor(n, 8, binding.GB_F64, A, n, Q, n, R, n, info), "qr host")
    Qo, Ro, _ = oracle.qr(A, 8)
    assert info[0] == 0
    assert np.abs(Q - Qo).max() <= 1e-12 and np.abs(R - Ro).max() <= 1e-12 * np.abs(Ro).max()
    assert h.gb_qr_factor(n, 8, binding.GB_F64, A, n, A, n, R, n, info) == -7  # Q overlaps A
    assert h.gb_qr_factor(n, 8, binding.GB_MIX_BF16, A, n, Q, n, R, n, info) == binding.GB_ERR_UNSUPPORTED
    assert h.gb_qr_factor(n, -1, binding.GB_F64, A, n, Q, n, R, n, info) == -3


def test_qr_zero_order(h):
    from paper_1812_02056_gb300 import binding
    info = torch.ones(1, dtype=torch.int32, device=DEV)
    binding.check(h.gb_qr_factor(0, 8, binding.GB_F64, None, 1, None, 1, None, 1, info), "n=0")
    assert int(info.item()) == 0
