"""Problem-level partition of a batch over the ranks of a multi-GPU job (host logic only).

The loop-shrinking path shards at problem granularity: every (mesh, seed vertex) problem -- its
initial pass, tunnel passes and refinement passes -- is independent of the others, while a single
front evolution is thousands of small band-local steps with global events and does not shard.  So
the problems of a batch are split over the ranks by a greedy longest-processing-time rule on their
face counts (the work of a problem grows with its mesh), each rank detects its share with one
batched call on its own GPU, and the per-problem results are gathered on rank 0 in the batch's
order.  The only exchange is that gather of results: no collective runs on the data path.
"""
from __future__ import annotations


def lpt_partition(weights, n_ranks: int) -> list:
    """Greedy LPT: items in order of decreasing weight (ties: smaller index first), each to the rank
    with the least total so far (ties: smaller rank).  Returns, per rank, its item indices in
    ascending order."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    load = [0.0] * n_ranks
    out = [[] for _ in range(n_ranks)]
    for i in sorted(range(len(weights)), key=lambda k: (-float(weights[k]), k)):
        r = min(range(n_ranks), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += float(weights[i])
    return [sorted(x) for x in out]


def flatten(problems) -> list:
    """(mesh index, seed) of every problem of a batch given as [(mesh, [seeds])], mesh-major,
    seed-minor (the library's problem order)."""
    return [(mi, s) for mi, (_, seeds) in enumerate(problems) for s in seeds]


def shard(problems, rank: int, n_ranks: int, faces=lambda m: m.nf):
    """This rank's share of a batch: (sub-batch as [(mesh, [seeds])], flat problem indices in the
    batch's order).  Weight of a problem: its mesh's face count."""
    flat = flatten(problems)
    parts = lpt_partition([faces(problems[mi][0]) for mi, _ in flat], n_ranks)
    mine = parts[rank]
    sub, last = [], None
    for i in mine:
        mi, s = flat[i]
        if mi != last:
            sub.append((problems[mi][0], []))
            last = mi
        sub[-1][1].append(s)
    return sub, mine


def gather(local_results, local_index, n_problems: int, dist=None):
    """Results of every rank's problems, on rank 0, in the batch's problem order (None on the other
    ranks).  local_results[k] is the result of flat problem local_index[k].  Without a process
    group, local_results must cover the whole batch."""
    pairs = list(zip(local_index, local_results))
    if dist is None:
        allp = [pairs]
    else:
        allp = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
        dist.gather_object(pairs, allp, dst=0)
        if dist.get_rank() != 0:
            return None
    out = [None] * n_problems
    for part in allp:
        for i, r in part:
            if out[i] is not None:
                raise RuntimeError(f"problem {i} came from two ranks")
            out[i] = r
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"problems {missing[:8]} came from no rank")
    return out


def detect_sharded(problems, detect, rank: int = 0, n_ranks: int = 1, dist=None):
    """Detect a batch over the ranks of a job: this rank runs detect(sub_batch) -> per-problem
    results on its share; rank 0 returns every result in batch order, other ranks None."""
    sub, mine = shard(problems, rank, n_ranks)
    local = detect(sub) if sub else []
    if len(local) != len(mine):
        raise RuntimeError(f"rank {rank}: {len(local)} results for {len(mine)} problems")
    return gather(local, mine, len(flatten(problems)), dist)
