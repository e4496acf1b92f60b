"""The continuous-batching server (gb_server_*).

* every result solves A X = B to FP64 backward error (host check);
* a job's result is the same bits alone and in a mix of concurrent jobs
  (its step depends on (n, dtype) only);
* admission respects the slot count and the memory budget, oversized jobs
  are rejected, a breaking-down job does not disturb the others, and a
  bounded wait reports a timeout.
"""
import numpy as np
import pytest

from paper_1812_02056_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def built():
    from paper_1812_02056_gb300 import _build, binding
    _build.build()
    return binding


def _job(n, nrhs, seed):
    A = I.spd_gram(n, seed, device=DEV)
    B = torch.from_numpy(I.rhs(n, nrhs, seed + 1)).to(DEV)
    X = torch.empty_like(B)
    return A, B, X


def _eta(A, X, B):
    R = B - A @ X
    den = A.abs().sum(1).max() * X.abs().max(0).values + B.abs().max(0).values
    return float((R.abs().max(0).values / den).max())


def test_server_results_are_fp64_accurate(built):
    srv = built.Server(0, 0, 3)
    jobs = []
    for i, (n, k, dt) in enumerate([(64, 1, "mix_bf16"), (200, 5, "f32"), (513, 16, "mix_f16"),
                                    (1000, 3, "f64"), (777, 64, "mix_bf16x3"), (1500, 2, "mix_bf16")]):
        A, B, X = _job(n, k, 100 + i)
        jobs.append((srv.submit(A, B, X, dtype=dt), A, B, X))
    for t, A, B, X in jobs:
        r = srv.wait(t)
        assert r.status == 0 and r.info == 0
        assert _eta(A, X, B) <= 2e-14
    st = srv.stats()
    assert st.completed == len(jobs) and st.p99_ms >= st.p50_ms > 0
    srv.close()


def test_server_result_same_alone_and_in_a_mix(built):
    srv = built.Server(0, 0, 4)
    A, B, X1 = _job(700, 8, 7)
    srv.wait(srv.submit(A, B, X1, dtype="mix_bf16"))
    others = [_job(n, 4, 50 + n) for n in (300, 1200, 90, 2000, 640, 1000, 150, 800)]
    X2 = torch.empty_like(X1)
    tickets = [srv.submit(*o, dtype="mix_bf16") for o in others[:4]]
    t_mid = srv.submit(A, B, X2, dtype="mix_bf16")
    tickets += [srv.submit(*o, dtype="mix_bf16") for o in others[4:]]
    for t in tickets:
        assert srv.wait(t).status == 0
    assert srv.wait(t_mid).status == 0
    assert torch.equal(X1, X2)
    assert srv.stats().max_running >= 2
    srv.close()


def test_server_admission_respects_slots_and_budget(built):
    srv = built.Server(0, 0, 2)
    jobs = [_job(n, 2, 9 + n) for n in (400, 900, 300, 1100, 500, 700)]
    ts = [srv.submit(*j, dtype="f32") for j in jobs]
    for t in ts:
        assert srv.wait(t).status == 0
    assert srv.stats().max_running <= 2
    srv.close()
    # a budget that holds one 1000-order FP32 job at a time serialises them
    # (footprint: FP64 A 8 MB + FP32 factor 4 MB + vectors + 8 MiB slack)
    srv = built.Server(0, 30_000_000, 4)
    jobs = [_job(1000, 2, 30 + i) for i in range(4)]
    ts = [srv.submit(*j, dtype="f32") for j in jobs]
    for t in ts:
        assert srv.wait(t).status == 0
    assert srv.stats().max_running == 1
    srv.close()


def test_server_rejects_oversized_jobs(built):
    srv = built.Server(0, 1 << 20, 2)
    A, B, X = _job(1000, 1, 3)
    with pytest.raises(built.GbError) as e:
        srv.submit(A, B, X, dtype="f32")
    assert e.value.status == built.GB_ERR_REJECTED
    assert srv.stats().rejected == 1
    srv.close()


def test_server_host_buffers(built):
    srv = built.Server(0, 0, 2)
    n, k = 321, 3
    A = I.spd_gram(n, 5)
    B = I.rhs(n, k, 6)
    X = np.zeros((n, k))
    r = srv.wait(srv.submit(A, B, X, dtype="mix_bf16"))
    assert r.status == 0
    assert np.abs(X - np.linalg.solve(A, B)).max() <= 1e-12 * np.abs(X).max()
    srv.close()


def test_server_breakdown_is_isolated(built):
    srv = built.Server(0, 0, 3)
    bad = _job(300, 2, 11)
    bad[0][150, 150] = -1e8
    good = [_job(n, 2, 12 + n) for n in (256, 512)]
    tb = srv.submit(*bad, dtype="f64")
    tg = [srv.submit(*g, dtype="f64") for g in good]
    rb = srv.wait(tb)
    assert rb.info == 151
    for t, (A, B, X) in zip(tg, good):
        r = srv.wait(t)
        assert r.status == 0 and r.info == 0 and _eta(A, X, B) <= 2e-14
    srv.close()


def test_server_bounded_wait(built):
    srv = built.Server(0, 0, 1)
    A, B, X = _job(4096, 4, 2)
    t = srv.submit(A, B, X, dtype="f64")
    with pytest.raises(built.GbError) as e:
        srv.wait(t, timeout_s=1e-4)
    assert e.value.status == built.GB_ERR_TIMEOUT
    assert srv.wait(t).status == 0
    srv.close()
