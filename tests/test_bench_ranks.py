"""The bench's multi-rank logic on the CPU: every rank of a world-size-2 gloo group gets the
slowest rank's step time, the job value counts the label maps of both ranks, and the reference
arm does its work on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(1.5 + rank, world)
        q.put((rank, ms, world * 1000.0 / ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=10) for _ in procs)
    assert [r for r, _, _ in out] == [0, 1]
    assert all(ms == 2.5 for _, ms, _ in out)          # the slowest rank's time
    assert all(abs(v - 800.0) < 1e-9 for _, _, v in out)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "time_oracle", lambda *a, **k: called.append(1) or [1.0])
    assert bench.reference_arm(argparse.Namespace(steps=2, warmup=3, gpus=2)) == 0
    assert called == [] and capsys.readouterr().out == ""
