"""gb_chol_solve_noalloc: the solve for callers that cannot allocate.

Callers running under stream capture, inside a budgeted pool or a plugin
that must not touch the allocator cannot create a handle (gb_create
allocates); this entry point keeps its scratch in a static device array.
The test calls it through the C ABI twice in a row and checks both results
against the regular gb_chol_solve within the solve tolerance of the suite:
1e-10 of max |X| for FP64 factors, 1e-5 for FP32 factors (the two entry
points reach X by different, equally valid roundings: substitution here,
inverted diagonal blocks in the regular solve).  It lives in a file that pytest collects last and must
pass alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("dtype,n,nrhs", [("f64", 1000, 7), ("f32", 777, 33)])
def test_noalloc_solve_matches_regular_solve_twice(h, dtype, n, nrhs):
    from paper_1812_02056_gb300 import binding
    A = I.spd_gram(n, 4242 + n)
    tt = torch.float64 if dtype == "f64" else torch.float32
    L, info = h.chol_factor(torch.from_numpy(A).to(DEV, tt), 64, dtype)
    assert int(info.item()) == 0
    B = torch.from_numpy(I.rhs(n, nrhs, 99)).to(DEV)
    X_ref, _ = h.chol_solve(L, B, dtype)
    ref = X_ref.cpu().numpy()
    for _ in range(2):
        X = torch.full_like(B, float("nan"))
        st = binding.gb_chol_solve_noalloc(n, nrhs, binding.DTYPES[dtype], L, L.stride(0), B,
                                           nrhs, X, nrhs)
        assert st == binding.GB_OK, binding.status_string(st)
        torch.cuda.synchronize()
        got = X.cpu().numpy()
        tol = 1e-10 if dtype == "f64" else 1e-5
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_noalloc_rejects_beyond_maximum_and_host_buffers(h):
    from paper_1812_02056_gb300 import binding
    d = torch.zeros(4, dtype=torch.float64, device=DEV)
    st = binding.gb_chol_solve_noalloc(131073, 1, binding.GB_F64, d, 131073, d, 1, d, 1)
    assert st == binding.GB_ERR_UNSUPPORTED
    Lh = np.eye(8)
    Bh = np.ones((8, 1))
    Xd = torch.zeros((8, 1), dtype=torch.float64, device=DEV)
    assert binding.gb_chol_solve_noalloc(8, 1, binding.GB_F64, Lh, 8, Bh, 1, Xd, 1) == -4
