"""Mixed-precision factorizations (FP32 working matrix, FP64 diagonal
blocks, tensor-core BF16/FP16 delayed update).

* Exact: the symmetric Pascal matrix of order 6 has entries <= 252 and a
  factor of small integers, all exact in BF16/FP16, so the mixed factor must
  equal the lower Pascal matrix bit for bit at every step s.
* Rounded: against the FP64 oracle the factor carries the error of 16-bit
  operands; bounds are stated per dtype (the unit roundoff 2^-8 for BF16 and
  2^-11 for FP16 times a small constant), on the normwise backward error and
  on the guarded elementwise error.
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests.helpers import guarded_rel_err, lu_split

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"

BOUNDS = {"mix_bf16": 2.0 ** -8 * 2, "mix_f16": 2.0 ** -11 * 2, "mix_bf16x3": 2.0 ** -22}


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
@pytest.mark.parametrize("s", [1, 2, 3])
def test_mixed_pascal_exact(h, dt, s):
    from paper_1812_02056_gb300 import binding
    h.set_option(binding.GB_OPT_INNER_STEP, 1)
    try:
        L, info = h.chol_factor(torch.from_numpy(I.pascal_sym(6)).to(DEV), s, dt)
    finally:
        h.set_option(binding.GB_OPT_INNER_STEP, 64)
    assert int(info.item()) == 0
    assert np.array_equal(L.double().cpu().numpy(), I.pascal_lower(6))


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
@pytest.mark.parametrize("n,s", [(512, 64), (700, 128), (1024, 256)])
def test_mixed_chol_vs_oracle(h, dt, n, s):
    A = I.spd_gram(n, 31 + n)
    L, info = h.chol_factor(torch.from_numpy(A).to(DEV), s, dt)
    assert int(info.item()) == 0
    Lg = L.double().cpu().numpy()
    be = oracle.chol_backward_error(A, Lg)
    assert be <= BOUNDS[dt]
    Lo, _ = oracle.chol(A, s)
    assert guarded_rel_err(Lg, Lo, floor=1e-2) <= 8 * BOUNDS[dt]


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16", "mix_bf16x3"])
def test_mixed_lu_vs_oracle(h, dt):
    n, s = 600, 128
    A = I.lu_diag_dominant(n, 77)
    LU, info = h.lu_factor(torch.from_numpy(A).to(DEV), s, dt)
    assert int(info.item()) == 0
    L, U = lu_split(LU.double().cpu().numpy())
    assert oracle.lu_backward_error(A, L, U) <= BOUNDS[dt]


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16"])
def test_mixed_matches_simt_update_closely(h, dt):
    """The tensor-core update and the FP32 CUDA-core update differ only by the
    16-bit rounding of the panel."""
    from paper_1812_02056_gb300 import binding
    n, s = 640, 128
    A = torch.from_numpy(I.spd_gram(n, 5)).to(DEV)
    L1, _ = h.chol_factor(A, s, dt)
    prev = h.get_option(binding.GB_OPT_TC_UPDATE)
    h.set_option(binding.GB_OPT_TC_UPDATE, 0)
    try:
        L2, _ = h.chol_factor(A, s, dt)
    finally:
        h.set_option(binding.GB_OPT_TC_UPDATE, prev)
    d = (L1.double() - L2.double()).abs().max().item() / L2.double().abs().max().item()
    assert d <= 4 * BOUNDS[dt]
