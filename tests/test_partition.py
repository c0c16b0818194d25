"""Problem-level partition of a batch over ranks (host logic, no GPU): greedy LPT on face counts,
the shard of each rank, and the gather of per-problem results on rank 0 -- in one process and over
world_size-2 gloo ranks with a stub detector."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2105_13168_gb300 import partition as pt  # noqa: E402


class M:
    def __init__(self, nf):
        self.nf = nf


def test_lpt_partition_rules():
    w = [7, 3, 3, 2, 2, 2, 1]
    parts = pt.lpt_partition(w, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(w)))
    loads = [sum(w[i] for i in p) for p in parts]
    # LPT: makespan within 4/3 of the optimum (here 7 = the largest item)
    assert max(loads) <= 4 / 3 * 7
    assert parts == pt.lpt_partition(w, 3)  # deterministic
    assert pt.lpt_partition(w, 1) == [list(range(len(w)))]
    # more ranks than items: the extra ranks get nothing
    assert pt.lpt_partition([5, 5], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        pt.lpt_partition(w, 0)


def test_shards_cover_the_batch_once():
    probs = [(M(100), [1, 2, 3, 4]), (M(7000), [5]), (M(40), [6, 7]), (M(900), [8, 9, 10])]
    flat = pt.flatten(probs)
    for n in (1, 2, 3, 5, 16):
        seen = []
        for r in range(n):
            sub, mine = pt.shard(probs, r, n)
            # the sub-batch lists exactly this rank's problems, mesh-major and in batch order
            assert [(mi, s) for mi, s in (flat[i] for i in mine)] == \
                [(next(k for k, (m, _) in enumerate(probs) if m is mm), s) for mm, ss in sub for s in ss]
            seen += mine
        assert sorted(seen) == list(range(len(flat)))


def test_gather_in_one_process():
    probs = [(M(10), [0, 1]), (M(20), [2])]
    out = pt.detect_sharded(probs, lambda sub: [f"r{s}" for _, ss in sub for s in ss])
    assert out == ["r0", "r1", "r2"]
    with pytest.raises(RuntimeError):
        pt.gather(["a"], [0], 2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2105_13168_gb300 import partition as p2

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        probs = [(M(50 * (i + 1)), [10 * i + k for k in range(3)]) for i in range(4)]

        def stub(sub):  # a detector: one result per problem, tagged with the rank that ran it
            return [{"seed": s, "nf": m.nf, "rank": rank} for m, ss in sub for s in ss]

        out = p2.detect_sharded(probs, stub, rank, world, dist)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_gather():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[1] is None
    out = res[0]
    assert [r["seed"] for r in out] == [10 * i + k for i in range(4) for k in range(3)]
    # both ranks worked, and their face totals are balanced by the LPT rule
    loads = {0: 0, 1: 0}
    for r in out:
        loads[r["rank"]] += r["nf"]
    assert loads[0] > 0 and loads[1] > 0
    assert max(loads.values()) <= 4 / 3 * (sum(loads.values()) / 2) + 200
