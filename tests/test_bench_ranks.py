"""Host logic of the multi-GPU benchmark on CPU: world_size-2 gloo ranks (no GPU).  Each rank
reports its own step time; the job's time is the slowest rank's and the whole-job value counts
the faces of every problem of the job (its problems partitioned over the ranks, weak scaling, no
collective on the data path)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist, "cpu")
        q.put((rank, ms_max, bench.whole_job_value(2_000_000 * world, ms_max)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in out] == [0, 1]
    for _, ms_max, value in out:
        assert ms_max == 150.0
        assert value == pytest.approx(2_000_000 * 2 / 0.150)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_value(1000, 500.0) == pytest.approx(2000.0)
    # the job at N GPUs: 4 N seeds of the tube chain, so each rank's LPT share is 4 problems
    from paper_2105_13168_gb300 import partition

    job = bench.job_problems(3, 0.1)
    assert len(job[0][1]) == 12 and len(set(job[0][1])) == 12
    assert [len(partition.shard(job, r, 3)[1]) for r in range(3)] == [4, 4, 4]
    assert bench.job_problems(1, 0.1)[0][1] == job[0][1][:4]
