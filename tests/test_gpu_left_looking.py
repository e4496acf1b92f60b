"""Left-looking tile accumulation for the tensor-core Cholesky
(GB_OPT_LEFT_LOOKING): each s-block column receives all earlier columns'
contributions in one product (K = the columns done) read from a resident
16-bit copy of L, instead of rank-s updates of the trailing matrix.

* A = L0 L0^T with L0 unit lower and entries in {-1, 0, 1}: every product
  and every partial sum is an exact small integer in BF16/FP16 and FP32, so
  both groupings give L0 bit for bit;
* random SPD: the backward error stays within the same dtype's bound as the
  right-looking path, and the two factors agree to the 16-bit rounding;
* the option falls back to the right-looking loop where it does not apply
  (FP64, s not a multiple of 64) and then changes nothing.
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"

BOUNDS = {"mix_bf16": 2.0 ** -8 * 2, "mix_f16": 2.0 ** -11 * 2}  # as for the right-looking path


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


def _factor(h, A, s, dt, left):
    from paper_1812_02056_gb300 import binding
    h.set_option(binding.GB_OPT_LEFT_LOOKING, 1 if left else 0)
    try:
        L, info = h.chol_factor(A, s, dt)
        torch.cuda.synchronize()
    finally:
        h.set_option(binding.GB_OPT_LEFT_LOOKING, 0)
    assert int(info.item()) == 0
    return L


def test_option_default_and_range(h):
    from paper_1812_02056_gb300 import binding
    assert h.get_option(binding.GB_OPT_LEFT_LOOKING) == 0
    h.set_option(binding.GB_OPT_LEFT_LOOKING, 1)
    assert h.get_option(binding.GB_OPT_LEFT_LOOKING) == 1
    h.set_option(binding.GB_OPT_LEFT_LOOKING, 0)


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16"])
@pytest.mark.parametrize("n,s", [(640, 128), (1024, 64), (1000, 256)])
def test_integer_factor_exact_both_groupings(h, dt, n, s):
    L0 = I.unit_lower_integer(n, 70 + n, -1, 1)
    A = torch.from_numpy(L0 @ L0.T).to(DEV)
    Ll = _factor(h, A, s, dt, True).double().cpu().numpy()
    Lr = _factor(h, A, s, dt, False).double().cpu().numpy()
    assert np.array_equal(Lr, L0)
    assert np.array_equal(Ll, L0)


@pytest.mark.parametrize("dt", ["mix_bf16", "mix_f16"])
@pytest.mark.parametrize("n,s", [(1024, 256), (2048, 128)])
def test_random_spd_within_bounds(h, dt, n, s):
    A = I.spd_gram(n, 80 + n)
    Ad = torch.from_numpy(A).to(DEV)
    Ll = _factor(h, Ad, s, dt, True).double().cpu().numpy()
    Lr = _factor(h, Ad, s, dt, False).double().cpu().numpy()
    assert oracle.chol_backward_error(A, Ll) <= BOUNDS[dt]
    assert oracle.chol_backward_error(A, Lr) <= BOUNDS[dt]
    d = np.abs(Ll - Lr).max() / np.abs(Lr).max()
    assert d <= 4 * BOUNDS[dt]


@pytest.mark.parametrize("dt,s", [("f64", 128), ("mix_bf16", 100), ("mix_bf16x3", 128)])
def test_fallback_is_the_right_looking_loop(h, dt, s):
    A = torch.from_numpy(I.spd_gram(500, 91)).to(DEV)
    Ll = _factor(h, A, s, dt, True)
    Lr = _factor(h, A, s, dt, False)
    assert torch.equal(Ll, Lr)
