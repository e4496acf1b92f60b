"""The N > 1 path of bench.py on CPU with two gloo ranks: every rank runs
its own replica (no data-path collective); the job's time is the max over
ranks and its value counts every rank's steps; the reference arm runs on
rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 150.0][rank]  # rank 1 is the slow replica
    mx = bench.dist_max(ms, dist, "cpu")
    val = bench.job_value(world, 10, 2e9, mx)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, val))


def test_two_gloo_ranks_max_time_and_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in out:
        assert mx == 150.0  # both ranks see the slowest replica's time
        # 2 ranks x 10 steps x 2 GFLOP in 0.15 s
        assert val == pytest.approx(2 * 10 * 2e9 / 0.150 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"n": 64, "s": 8, "steps": 1, "warmup": 0, "gpus": 2, "ref_n": 64})()
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_max(3.5) == 3.5
    assert bench.job_value(1, 4, 1e9, 2000.0) == pytest.approx(2.0)
