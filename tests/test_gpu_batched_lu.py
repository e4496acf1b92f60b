"""Batched Algorithm 2 (pivot-free Crout LU): one persistent launch over many
uneven matrices (gb_lu_factor_batched).

* FP64 with GB_OPT_BATCHED_EXACT (no FMA): the compact factor of every matrix
  is the same bits as the oracle's L and strict upper U at the same step s,
  in the shared-memory path (FP64 n <= 118) and in the panel path.
* A = L0 U0 with small-integer unit-diagonal factors: every operation is
  exact, so both arithmetic modes recover L0 and U0 exactly (closed form).
* FP32 against the oracle on the FP32-rounded input.
* per-matrix breakdown (L_cc = 0) in both paths, out-of-place with padded
  leading dimensions, and CUDA-graph capture of the plan.
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


def _step_used(n, s, esz):
    """Step a matrix of order n runs with (the rule stated in gbchol.h)."""
    elems = 110 * 1024 // esz
    ld = n if n % 2 else n + 1
    if n * ld <= elems:
        return min(s, n)
    return max(1, min(s, elems // (2 * n)))


def _mats(sizes, seed, dtype=torch.float64):
    return [torch.from_numpy(I.lu_diag_dominant(int(n), seed + i)).to(DEV, dtype)
            for i, n in enumerate(sizes)]


def _oracle_compact(A, s):
    L, U, info = oracle.lu(A, s)
    return np.tril(L) + np.triu(U, 1), info


SIZES = [1, 2, 3, 7, 16, 33, 64, 100, 117, 118, 119, 150, 167, 168, 200, 300, 512]


def test_step_rule():
    assert _step_used(118, 64, 8) == 64 and _step_used(119, 64, 8) == 59
    assert _step_used(167, 100, 4) == 100 and _step_used(168, 100, 4) == 83


@pytest.mark.parametrize("s", [1, 5, 32])
def test_batched_lu_fp64_exact_matches_oracle_bitwise(h, s):
    from paper_1812_02056_gb300 import binding
    mats = _mats(SIZES, 100 + s)
    host = [m.cpu().numpy().copy() for m in mats]
    h.set_option(binding.GB_OPT_BATCHED_EXACT, 1)
    try:
        info = h.lu_factor_batched(mats, s=s, dtype="f64")
    finally:
        h.set_option(binding.GB_OPT_BATCHED_EXACT, 0)
    assert np.all(info == 0)
    for A, m in zip(host, mats):
        ref, io = _oracle_compact(A, _step_used(A.shape[0], s, 8))
        assert io == 0
        assert np.array_equal(m.cpu().numpy(), ref), A.shape[0]


@pytest.mark.parametrize("s", [8, 32])
def test_batched_lu_fp64_fma_within_tolerance(h, s):
    mats = _mats(SIZES, 200)
    host = [m.cpu().numpy().copy() for m in mats]
    info = h.lu_factor_batched(mats, s=s, dtype="f64")
    assert np.all(info == 0)
    for A, m in zip(host, mats):
        ref, _ = _oracle_compact(A, s)
        got = m.cpu().numpy()
        assert guarded_rel_err(got, ref) <= 1e-10
        L, U = lu_split(got)
        assert oracle.lu_backward_error(A, L, U) <= 1e-14


@pytest.mark.parametrize("exact", [0, 1])
def test_batched_lu_integer_factors_exact(h, exact):
    """A = L0 U0, L0 unit lower and U0 unit upper with entries in {-1, 0, 1}:
    every intermediate is a small integer, so L = L0 and U = U0 exactly."""
    from paper_1812_02056_gb300 import binding
    sizes = [5, 64, 118, 119, 250, 400]
    mats, want = [], []
    for i, n in enumerate(sizes):
        L0 = I.unit_lower_integer(n, 300 + i, -1, 1)
        U0 = I.unit_lower_integer(n, 400 + i, -1, 1).T
        mats.append(torch.from_numpy(L0 @ U0).to(DEV))
        want.append(np.tril(L0) + np.triu(U0, 1))
    h.set_option(binding.GB_OPT_BATCHED_EXACT, exact)
    try:
        info = h.lu_factor_batched(mats, s=16, dtype="f64")
    finally:
        h.set_option(binding.GB_OPT_BATCHED_EXACT, 0)
    assert np.all(info == 0)
    for m, w in zip(mats, want):
        assert np.array_equal(m.cpu().numpy(), w)


@pytest.mark.parametrize("s", [4, 32, 64])
def test_batched_lu_fp32(h, s):
    mats = _mats(SIZES + [319, 320, 400], 500, torch.float32)
    host = [m.double().cpu().numpy().copy() for m in mats]
    info = h.lu_factor_batched(mats, s=s, dtype="f32")
    assert np.all(info == 0)
    for A, m in zip(host, mats):
        got = m.double().cpu().numpy()
        ref, _ = _oracle_compact(A, s)
        assert guarded_rel_err(got, ref, floor=1e-2) <= 2e-4
        L, U = lu_split(got)
        assert oracle.lu_backward_error(A, L, U) <= 2e-6


def test_batched_lu_breakdown_is_per_matrix(h):
    """L0 with a zero at diagonal k (and U0 unit upper, integer): the Crout
    recursion meets L_kk = 0 exactly, so info = k + 1."""
    sizes, ks = [40, 300, 60, 250], [None, 137, 0, None]
    mats = []
    for i, (n, k) in enumerate(zip(sizes, ks)):
        L0 = I.unit_lower_integer(n, 600 + i, -1, 1)
        if k is not None:
            L0[k, k] = 0.0
        U0 = I.unit_lower_integer(n, 700 + i, -1, 1).T
        mats.append(torch.from_numpy(L0 @ U0).to(DEV))
    info = h.lu_factor_batched(mats, s=16, dtype="f64")
    assert list(info) == [0, 138, 1, 0]


def test_batched_lu_out_of_place_and_padded(h):
    sizes = [37, 230, 5]
    mats = _mats(sizes, 800)
    padded = []
    for m in mats:
        n = m.shape[0]
        big = torch.full((n, n + 3), 7.0, dtype=torch.float64, device=DEV)
        big[:, :n] = m
        padded.append(big[:, :n])
    out_big = [torch.full((m.shape[0], m.shape[0] + 1), 9.0, dtype=torch.float64, device=DEV)
               for m in mats]
    outs = [b[:, :m.shape[0]] for b, m in zip(out_big, mats)]
    before = [p.clone() for p in padded]
    info = h.lu_factor_batched(padded, s=8, dtype="f64", outs=outs)
    assert np.all(info == 0)
    for p, b in zip(padded, before):
        assert torch.equal(p, b)
    for m, o, b in zip(mats, outs, out_big):
        ref, _ = _oracle_compact(m.cpu().numpy(), 8)
        assert guarded_rel_err(o.cpu().numpy(), ref) <= 1e-10
        assert bool((b[:, m.shape[0]:] == 9.0).all())


def test_batched_lu_graph_capture_and_replay(h):
    from paper_1812_02056_gb300 import binding
    sizes = [64, 128, 300, 17, 200] * 3
    mats = _mats(sizes, 900)
    outs = [torch.empty_like(m) for m in mats]
    cnt = len(mats)
    n_arr = np.array(sizes, dtype=np.int64)
    a_arr = np.array([m.data_ptr() for m in mats], dtype=np.uint64)
    l_arr = np.array([o.data_ptr() for o in outs], dtype=np.uint64)
    binding.check(h.gb_lu_batched_plan(cnt, n_arr, a_arr, n_arr, l_arr, n_arr, binding.GB_F64,
                                       16), "plan")
    info = torch.ones(cnt, dtype=torch.int32, device=DEV)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        binding.check(h.gb_batched_run(info, s), "warm run")
    torch.cuda.synchronize()
    for m, o in zip(mats, outs):
        ref, _ = _oracle_compact(m.cpu().numpy(), 16)
        assert guarded_rel_err(o.cpu().numpy(), ref) <= 1e-10
    ref = [o.clone() for o in outs]
    with torch.cuda.graph(g, stream=s):
        binding.check(h.gb_batched_run(info, s), "captured run")
    for _ in range(2):
        for o in outs:
            o.fill_(3.0)
        g.replay()
        torch.cuda.synchronize()
        assert int(info.abs().sum().item()) == 0
        for o, r in zip(outs, ref):
            assert torch.equal(o, r)


def test_batched_lu_empty_and_zero_order(h):
    from paper_1812_02056_gb300 import binding
    assert h.lu_factor_batched([], s=8, dtype="f64").size == 0
    mats = [torch.zeros((0, 0), dtype=torch.float64, device=DEV),
            torch.from_numpy(I.lu_diag_dominant(9, 3)).to(DEV)]
    host = mats[1].cpu().numpy().copy()
    info = h.lu_factor_batched(mats, s=4, dtype="f64")
    assert list(info) == [0, 0]
    ref, _ = _oracle_compact(host, 4)
    assert guarded_rel_err(mats[1].cpu().numpy(), ref) <= 1e-12
    st = h.gb_lu_factor_batched(1, np.array([2000], dtype=np.int64),
                                np.array([mats[1].data_ptr()], dtype=np.uint64),
                                np.array([2000], dtype=np.int64),
                                np.array([mats[1].data_ptr()], dtype=np.uint64),
                                np.array([2000], dtype=np.int64), binding.GB_F64, 4, None)
    assert st == -3  # order above the batched maximum (1024)
