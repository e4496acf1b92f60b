"""Batched Algorithm 1: one persistent launch over many uneven matrices.

* FP64 with GB_OPT_BATCHED_EXACT (every product and subtraction rounded
  separately, no FMA): the factor of every matrix is the same bits as the
  oracle's literal mode at the same step s -- both in the shared-memory path
  and in the panel path.
* FP32: the oracle on the FP32-rounded input, FP32 bounds of the suite.
* per-matrix breakdown columns, out-of-place operation, padded leading
  dimensions, CUDA-graph capture and replay, the step autotuner, and a
  sample of the 10,000-matrix workload.
"""
import numpy as np
import pytest

import oracle
from paper_1812_02056_gb300 import inputs as I
from tests.helpers import guarded_rel_err

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
    if n * (n + 1) // 2 <= elems:
        return min(s, n)
    return max(1, min(s, elems // n))


def _mats(sizes, seed, dtype=torch.float64):
    buf, offs = I.batch_spd_device(sizes, seed, DEV, dtype)
    return [buf[o:o + n * n].view(n, n) for o, n in zip(offs, sizes)]


SIZES = [1, 2, 3, 7, 16, 33, 64, 100, 150, 167, 168, 200, 236, 237, 260, 300, 512]


@pytest.mark.parametrize("s", [1, 5, 32])
def test_batched_fp64_exact_matches_oracle_bitwise(h, s):
    from paper_1812_02056_gb300 import binding
    mats = _mats(SIZES, 11 + s)
    host = [m.cpu().numpy().copy() for m in mats]
    h.set_option(binding.GB_OPT_BATCHED_EXACT, 1)
    try:
        info = h.chol_factor_batched(mats, s=s, dtype="f64")
    finally:
        h.set_option(binding.GB_OPT_BATCHED_EXACT, 0)
    assert np.all(info == 0)
    for A, m in zip(host, mats):
        Lo, io = oracle.chol(A, _step_used(A.shape[0], s, 8))
        assert io == 0
        assert np.array_equal(m.cpu().numpy(), Lo), A.shape[0]


@pytest.mark.parametrize("s", [8, 32])
def test_batched_fp64_fma_within_tolerance(h, s):
    mats = _mats(SIZES, 21)
    host = [m.cpu().numpy().copy() for m in mats]
    info = h.chol_factor_batched(mats, s=s, dtype="f64")
    assert np.all(info == 0)
    for A, m in zip(host, mats):
        Lo, _ = oracle.chol(A, s)
        assert guarded_rel_err(m.cpu().numpy(), Lo) <= 1e-10


@pytest.mark.parametrize("s", [4, 32, 64])
def test_batched_fp32(h, s):
    mats = _mats(SIZES + [319, 320, 400], 31, torch.float32)
    host = [m.double().cpu().numpy().copy() for m in mats]
    info = h.chol_factor_batched(mats, s=s, dtype="f32")
    assert np.all(info == 0)
    for A, m in zip(host, mats):
        L = m.double().cpu().numpy()
        Lo, _ = oracle.chol(A, s)
        assert guarded_rel_err(L, Lo, floor=1e-2) <= 2e-4
        assert oracle.chol_backward_error(A, L) <= 2e-6


def test_batched_breakdown_is_per_matrix(h):
    sizes = [50, 300, 40, 250]
    mats = _mats(sizes, 5)
    mats[1][123, 123] = -1.0e9
    mats[2][0, 0] = float("nan")
    info = h.chol_factor_batched(mats, s=16, dtype="f64")
    assert info[0] == 0 and info[3] == 0
    assert info[1] == 124 and info[2] == 1


def test_batched_out_of_place_and_padded(h):
    from paper_1812_02056_gb300 import binding
    sizes = [37, 230, 5]
    mats = _mats(sizes, 8)
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
    info = h.chol_factor_batched(padded, s=8, dtype="f64", outs=outs)
    assert np.all(info == 0)
    for p, b in zip(padded, before):
        assert torch.equal(p, b)  # inputs untouched
    for m, o, b in zip(mats, outs, out_big):
        Lo, _ = oracle.chol(m.cpu().numpy(), 8)
        assert guarded_rel_err(o.cpu().numpy(), Lo) <= 1e-10
        assert bool((b[:, m.shape[0]:] == 9.0).all())  # padding untouched


def test_batched_graph_capture_and_replay(h):
    from paper_1812_02056_gb300 import binding
    sizes = [64, 128, 300, 17, 200] * 3
    mats = _mats(sizes, 9)
    outs = [torch.empty_like(m) for m in mats]
    cnt = len(mats)
    n_arr = np.array(sizes, dtype=np.int64)
    a_arr = np.array([m.data_ptr() for m in mats], dtype=np.uint64)
    l_arr = np.array([o.data_ptr() for o in outs], dtype=np.uint64)
    binding.check(h.gb_batched_plan(cnt, n_arr, a_arr, n_arr, l_arr, n_arr, binding.GB_F64, 16),
                  "plan")
    info = torch.ones(cnt, dtype=torch.int32, device=DEV)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        binding.check(h.gb_batched_run(info, s), "warm run")
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
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


def test_batched_autotune_then_default_steps(h):
    from paper_1812_02056_gb300 import binding
    steps = np.zeros(8, dtype=np.int32)
    binding.check(h.gb_batched_tune(binding.GB_F32, 256, steps), "tune")
    assert np.all(steps >= 1)
    mats = _mats([20, 100, 250], 4, torch.float32)
    host = [m.double().cpu().numpy().copy() for m in mats]
    info = h.chol_factor_batched(mats, s=0, dtype="f32")
    assert np.all(info == 0)
    for A, m in zip(host, mats):
        assert oracle.chol_backward_error(A, m.double().cpu().numpy()) <= 2e-6


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_10000_matrices_sampled(h, dtype):
    """The batched workload at full size: 10,000 SPD matrices, n uniform on
    [16, 512], one launch; every info is 0 and a sample matches the oracle."""
    sizes = I.batch_sizes(10000, 16, 512, I.seed_for(I.W_BATCHED))
    tt = torch.float64 if dtype == "f64" else torch.float32
    buf, offs = I.batch_spd_device(sizes, I.seed_for(I.W_BATCHED, 1), DEV, tt)
    mats = [buf[o:o + n * n].view(n, n) for o, n in zip(offs, sizes)]
    rng = np.random.default_rng(0)
    pick = rng.choice(len(sizes), 12, replace=False)
    host = {int(i): mats[i].double().cpu().numpy().copy() for i in pick}
    outs = [torch.empty_like(m) for m in mats]
    info = h.chol_factor_batched(mats, s=32, dtype=dtype, outs=outs)
    assert np.all(info == 0)
    for i, A in host.items():
        L = outs[i].double().cpu().numpy()
        Lo, _ = oracle.chol(A, 32)
        if dtype == "f64":
            assert guarded_rel_err(L, Lo) <= 1e-10
            assert oracle.chol_backward_error(A, L) <= 1e-13
        else:
            assert guarded_rel_err(L, Lo, floor=1e-2) <= 2e-4
