"""The step autotuner (gb_tune_step) and s = 0 after tuning.

The tuner times candidate (s, inner step) pairs on n I + ones and keeps the
fastest for the order's power-of-two range; a factorization called with
s = 0 then runs with that pair.  The results must still be the method's:
checked against the oracle at the tuned s (Cholesky, LU: FP64 tolerance;
QR: Gram-Schmidt's 10 n u cond(A)).  The handle's own inner step is left as
it was.
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


def test_tune_chol_then_default_step(h):
    from paper_1812_02056_gb300 import binding
    n = 1024
    inner_before = h.get_option(binding.GB_OPT_INNER_STEP)
    s, b = h.tune_step("chol", "f64", n)
    assert s in (32, 64, 128, 256, 512) and b in (16, 32, 64) and b <= s
    assert h.get_option(binding.GB_OPT_INNER_STEP) == inner_before
    A = I.spd_gram(800, 3)       # in [512, 1024): not tuned, the default step
    A2 = I.spd_gram(n + 100, 4)  # in [1024, 2048): the tuned pair
    L, info = h.chol_factor(torch.from_numpy(A2).to(DEV), 0, "f64")
    assert int(info.item()) == 0
    Lo, _ = oracle.chol(A2, s)
    assert guarded_rel_err(L.cpu().numpy(), Lo) <= 1e-10
    L1, info1 = h.chol_factor(torch.from_numpy(A).to(DEV), 0, "f64")  # untuned range: default
    assert int(info1.item()) == 0
    assert oracle.chol_backward_error(A, L1.cpu().numpy()) <= 1e-14


def test_tune_lu_mixed(h):
    n = 600
    s, b = h.tune_step("lu", "mix_bf16x3", n)
    assert s in (32, 64, 128, 256, 512) and b <= s
    A = I.lu_diag_dominant(n, 8)
    LU, info = h.lu_factor(torch.from_numpy(A).to(DEV), 0, "mix_bf16x3")
    assert int(info.item()) == 0
    L, U = lu_split(LU.double().cpu().numpy())
    assert oracle.lu_backward_error(A, L, U) <= 1e-6


def test_tune_qr(h):
    from paper_1812_02056_gb300 import binding
    n = 512
    s, b = h.tune_step("qr", "f64", n)
    assert s in (32, 64, 128, 256) and b in (8, 16, 32) and b <= s
    assert h.get_option(binding.GB_OPT_QR_INNER_STEP) == 16
    A = I.gaussian(n, n, 9) + 2.0 * np.sqrt(n) * np.eye(n)
    Qd, Rd, info = h.qr_factor(torch.from_numpy(A).to(DEV), 0, "f64")
    assert int(info.item()) == 0
    Qo, Ro, _ = oracle.qr(A, s)
    tol = 10 * n * 2.0 ** -53 * np.linalg.cond(A)
    assert np.abs(Qd.cpu().numpy() - Qo).max() <= tol


def test_tune_rejections(h):
    from paper_1812_02056_gb300 import binding
    lib = h.lib
    assert lib.gb_tune_step(h.h, 3, binding.GB_F64, 100, None, None, None) == -2
    assert lib.gb_tune_step(h.h, 0, 9, 100, None, None, None) == -3
    assert lib.gb_tune_step(h.h, 0, binding.GB_F64, 1, None, None, None) == -4
    assert lib.gb_tune_step(h.h, 2, binding.GB_MIX_BF16, 100, None, None, None) == \
        binding.GB_ERR_UNSUPPORTED
