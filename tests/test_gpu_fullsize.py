"""Parity at the full benchmark sizes (n = 8192), in the launch
configuration bench.py times (FP64, s = 256, inner step 64, the same seeded
input): the whole factor against the oracle's, plus the pivot-free LU and the
FP32 factor on their leading blocks (the leading k x k block of a factor
depends only on the leading k x k block of A) and the device backward error.
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests.helpers import guarded_rel_err, lu_split, row_scaled_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
N = 8192


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


@pytest.fixture(scope="module")
def spd():
    A = I.spd_gram(N, I.seed_for(I.W_N8192, 0), device=DEV)  # bench.py's rank-0 input
    return A


def test_chol_f64_n8192_s256_full_oracle(h, spd):
    L, info = h.chol_factor(spd, 256, "f64")
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    be = h.backward_error(spd, L, "f64")
    assert be <= 1e-13
    Ah = spd.cpu().numpy()
    Lg = L.cpu().numpy()
    assert np.all(np.triu(Lg, 1) == 0.0)
    Lo, info_o = oracle.chol(Ah, 256)
    assert info_o == 0
    assert guarded_rel_err(Lg, Lo) <= 1e-10


@pytest.mark.parametrize("s", [117, 512])
def test_chol_f64_n8192_other_steps(h, spd, s):
    L, info = h.chol_factor(spd, s, "f64")
    assert int(info.item()) == 0
    assert h.backward_error(spd, L, "f64") <= 1e-13
    k = 1024
    Ah = spd[:k, :k].cpu().numpy()
    Lo, _ = oracle.chol(Ah, s)
    assert guarded_rel_err(L[:k, :k].cpu().numpy(), Lo) <= 1e-10


def test_chol_f32_n8192(h, spd):
    """FP32 at full size.  The leading 1024 x 1024 block of the factor
    depends only on the leading block of A: its backward error is taken by
    the oracle, and each entry is compared with the oracle's in units of the
    FP32 rounding model (tests.helpers.row_scaled_err, u = 2^-24; measured
    maxima are a few units)."""
    A32 = spd.float()
    L, info = h.chol_factor(A32, 256, "f32")
    assert int(info.item()) == 0
    assert h.backward_error(A32.double(), L, "f32") <= 2e-6
    k = 1024
    Ah = A32[:k, :k].double().cpu().numpy()
    Lk = L[:k, :k].double().cpu().numpy()
    assert oracle.chol_backward_error(Ah, Lk) <= 8 * np.sqrt(k) * 2.0 ** -24
    Lo, _ = oracle.chol(Ah, 256)
    e = row_scaled_err(Lk, Lo, 2.0 ** -24)
    assert e <= 16.0, f"row-scaled error {e:.2f}"


def test_lu_f64_n8192(h):
    A = torch.from_numpy(I.lu_diag_dominant(N, I.seed_for(I.W_N8192, 50))).to(DEV)
    LU, info = h.lu_factor(A, 256, "f64")
    assert int(info.item()) == 0
    assert h.backward_error(A, LU, "f64", lu=True) <= 1e-13
    k = 1024
    Lo, Uo, _ = oracle.lu(A[:k, :k].cpu().numpy(), 256)
    L, U = lu_split(LU[:k, :k].cpu().numpy())
    assert guarded_rel_err(L, Lo) <= 1e-10 and guarded_rel_err(U, Uo) <= 1e-10
