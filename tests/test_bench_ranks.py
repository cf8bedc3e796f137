"""bench.py's multi-rank logic on CPU: world_size 2 over gloo.  The ranks
share one job (each renders a shard of its words); the job's time is the
slowest rank's, and value counts the job's words once.  The reference arm
runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        barrier = bench.make_barrier(world)
        barrier()
        local_ms = [40.0, 55.0][rank]           # rank 1 is the slow one
        value, job_ms = bench.job_rate(1000, 10, local_ms,
                                       bench.make_max_over_ranks(world, "cpu"))
        out[rank] = (value, job_ms)
        barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_job_rate():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    value, job_ms = res[0]
    assert job_ms == 55.0
    assert value == pytest.approx(1000 * 10 / 0.055)


def test_single_rank_rate_needs_no_process_group():
    value, job_ms = bench.job_rate(516560652, 50, 20.0, bench.make_max_over_ranks(1, "cpu"))
    assert job_ms == 20.0 and value == pytest.approx(516560652 * 50 / 0.020)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import sys
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1",
                                      "--warmup", "1"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""
