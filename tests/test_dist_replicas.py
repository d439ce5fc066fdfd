"""Multi-GPU form of this build: replicas.  Each GPU solves its own copy of
the workload with no data exchange; the job is timed by its slowest rank
and its throughput is every rank's solves over that time.  The host-side
logic of bench.py is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 10.0 * (rank + 1)          # rank 1 is the slow one
        m = bench.max_over_ranks(ms)
        q.put((rank, m, bench.whole_job_rate(30.0, world, m)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_slowest_rank_and_whole_job_rate():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in out:
        assert m == 20.0                       # max over ranks on every rank
        assert rate == pytest.approx(30.0 * 2 / 0.020)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(3.0, 1, 10.0) == pytest.approx(300.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the other ranks exit without work or output."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "oracle_case", lambda: called.append(1))
    bench.run_reference(type("A", (), {"warmup": 1, "steps": 1})())
    assert not called and capsys.readouterr().out == ""
