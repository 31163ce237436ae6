"""The replica (N > 1) path of bench.py on CPU: two gloo ranks, each with its
own timings, agree on the element-wise maximum, and the whole-job value is
world x per-rank work / slowest time.  The reference arm prints on rank 0
only."""
import contextlib
import io
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [1.0 + rank, 5.0 - rank]                  # rank 0: (1, 5); rank 1: (2, 4)
        got = bench.max_over_ranks(mine, dist, "cpu")
        dist.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1] == [2.0, 5.0]


def test_whole_job_value_is_weak_scaling():
    # 4 replicas of 2048^2 nodes, 100 steps, slowest rank 0.011 s
    v = bench.whole_job_mlups(2048 * 2048, 100, 4, 0.011)
    assert v == pytest.approx(4 * 2048 * 2048 * 100 / 0.011 / 1e6)


def test_reference_arm_is_silent_off_rank0(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 3, 3, 2

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A())
    assert buf.getvalue() == ""
