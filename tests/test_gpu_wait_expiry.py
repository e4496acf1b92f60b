"""A bounded device wait that runs out, on the GPU, without any fault.

The single-launch triangular solve orders its blocks by a progress word:
each block waits (bounded by GB_OPT_SPIN_LIMIT, read from %globaltimer) for
the block before it to publish.  The test hook GB_OPT_TEST_WITHHOLD makes one
block of the forward sweep skip its publication, so the next block's wait
runs out: it raises the timeout word and returns, every later block sees the
word and returns, and the call reports GB_ERR_TIMEOUT within a few limits.
The next call on the same handle must then succeed and match the oracle:
its sync words start fresh and the timeout word was cleared.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
LIMIT = 20000  # x 100 ns = 2 ms


@pytest.fixture(scope="module")
def h():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    hd = binding.Handle(0)
    yield hd
    hd.close()


def test_option_default_and_range(h):
    from paper_1812_02056_gb300 import binding
    assert h.get_option(binding.GB_OPT_TEST_WITHHOLD) == 0
    assert h.lib.gb_set_option(h.h, binding.GB_OPT_TEST_WITHHOLD, -1) == -3
    h.set_option(binding.GB_OPT_TEST_WITHHOLD, 3)
    assert h.get_option(binding.GB_OPT_TEST_WITHHOLD) == 3
    h.set_option(binding.GB_OPT_TEST_WITHHOLD, 0)


def _withheld(h, fn, *a):
    from paper_1812_02056_gb300 import binding
    spin = h.get_option(binding.GB_OPT_SPIN_LIMIT)
    h.set_option(binding.GB_OPT_SPIN_LIMIT, LIMIT)
    h.set_option(binding.GB_OPT_TEST_WITHHOLD, 5)
    try:
        t0 = time.perf_counter()
        st, stats = fn(*a)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
    finally:
        h.set_option(binding.GB_OPT_TEST_WITHHOLD, 0)
        h.set_option(binding.GB_OPT_SPIN_LIMIT, spin)
    return st, stats, el


@pytest.mark.parametrize("dtype,refine", [("f64", False), ("f32", False), ("f32", True)])
def test_chol_solve_wait_expires_then_recovers(h, dtype, refine):
    from paper_1812_02056_gb300 import binding
    n, nrhs = 4096, 4
    A = I.spd_gram(n, 9300)
    Ad = torch.from_numpy(A).to(DEV)
    tt = torch.float64 if dtype == "f64" else torch.float32
    L, info = h.chol_factor(Ad.to(tt), 128, dtype)
    assert int(info.item()) == 0
    Bn = I.rhs(n, nrhs, 9301)
    B = torch.from_numpy(Bn).to(DEV)
    X = torch.empty_like(B)
    dt = binding.DTYPES[dtype]
    Aref = Ad if refine else None
    st, stats, el = _withheld(h, h.gb_chol_solve, n, nrhs, dt, L, n, Aref, n, B, nrhs, X, nrhs)
    assert st == binding.GB_ERR_TIMEOUT, binding.status_string(st)
    assert el < 5.0  # a few 2 ms limits, not the default 6.7 s
    if refine:
        assert stats.converged == 0
    # the same handle, the default limit, no hook: a normal solve
    st, stats = h.gb_chol_solve(n, nrhs, dt, L, n, Aref, n, B, nrhs, X, nrhs)
    torch.cuda.synchronize()
    assert st == binding.GB_OK, binding.status_string(st)
    if refine:  # refined to FP64 accuracy: against the oracle's FP64 solve
        Lo, _ = oracle.chol(A, 128)
        Xo = oracle.chol_solve(Lo, Bn)
        assert stats.eta <= 1e-14
    else:  # plain substitution with the factor itself
        Xo = oracle.chol_solve(np.tril(L.double().cpu().numpy()), Bn)
    tol = 1e-10 if (dtype == "f64" or refine) else 1e-5
    assert np.abs(X.cpu().numpy() - Xo).max() <= tol * np.abs(Xo).max()


def test_lu_solve_wait_expires_then_recovers(h):
    from paper_1812_02056_gb300 import binding
    n, nrhs = 2048, 3
    C = I.lu_diag_dominant(n, 9302)
    LU, info = h.lu_factor(torch.from_numpy(C).to(DEV), 128, "f64")
    assert int(info.item()) == 0
    Bn = I.rhs(n, nrhs, 9303)
    B = torch.from_numpy(Bn).to(DEV)
    X = torch.empty_like(B)
    st, _, el = _withheld(h, h.gb_lu_solve, n, nrhs, binding.GB_F64, LU, n, None, n, B, nrhs, X,
                          nrhs)
    assert st == binding.GB_ERR_TIMEOUT and el < 5.0
    st, _ = h.gb_lu_solve(n, nrhs, binding.GB_F64, LU, n, None, n, B, nrhs, X, nrhs)
    torch.cuda.synchronize()
    assert st == binding.GB_OK
    F = LU.cpu().numpy()
    Xo = oracle.lu_solve(np.tril(F), np.triu(F, 1) + np.eye(n), Bn)
    assert np.abs(X.cpu().numpy() - Xo).max() <= 1e-10 * np.abs(Xo).max()
