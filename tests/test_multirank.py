"""The multi-replica path of bench.py on CPU: two gloo ranks (the GPU run
uses NCCL with the same calls).  The job's time is the slowest rank's, the
value counts every rank's work, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        ms, gbs = bench.job_throughput(10.0 * (rank + 1), 1e9, 2, world)
        q.put((rank, ms, gbs))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_both():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, gbs in got:
        assert ms == 20.0  # the slower rank's 20 ms
        assert gbs == pytest.approx(2 * 2 * 1e9 / 0.020 / 1e9)  # both ranks' bytes


def test_single_rank_needs_no_process_group():
    import bench
    ms, gbs = bench.job_throughput(5.0, 2e9, 3, 1)
    assert ms == 5.0 and gbs == pytest.approx(3 * 2e9 / 0.005 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    rc = bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=0))
    assert rc == 0 and capsys.readouterr().out == ""
