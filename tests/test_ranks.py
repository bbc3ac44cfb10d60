"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): views
are independent, so ranks run replicas and only the timing is combined --
the job's step time is the slowest rank's and the job's rate is the ranks'
frames over it.  Also: the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        local_ms = [2.0, 3.5][rank]               # rank 1 is the slow one
        ms = bench.max_over_ranks(torch, dist, local_ms, world, "cpu")
        q.put((rank, ms, bench.job_rate(ms, world)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in res:
        assert ms == 3.5
        assert rate == pytest.approx(2 * 1000.0 / 3.5)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(torch, None, 1.25, 1, "cpu") == 1.25
    assert bench.job_rate(2.0, 1) == 500.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "cpu_oracle_fps", lambda *a, **k: called.append(1))
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.reference_arm(args)
    assert called == [] and capsys.readouterr().out == ""
