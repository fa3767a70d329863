"""Independent systems spread over the ranks of a process group, one GPU per rank.

A batch of systems A_i x_i = b_i has no exchange step: each rank solves a subset on its own GPU
(through the CUDA library) and the results are gathered. The subsets balance the O(n^3)
factorization work by the longest-processing-time rule. A single system does not shard (its LU
and Arnoldi products are not split); several GPUs then run independent replicas, and a timing is
the maximum over the ranks.

Host logic only: the process group may be NCCL (GPU ranks) or gloo (CPU, for tests); nothing here
computes a step of the method.
"""
from __future__ import annotations


def shard_by_work(sizes, world):
    """Indices of the systems each rank solves: the largest n first, each to the rank with the
    least n^3 so far (ties to the lower rank). One sorted index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    loads = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i)):
        r = min(range(world), key=lambda q: (loads[q], q))
        out[r].append(i)
        loads[r] += float(sizes[i]) ** 3
    return [sorted(o) for o in out]


def _group():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def max_over_ranks(value, device=None):
    """The maximum of a number over the ranks of the default process group (the number itself
    without a group). device: where the reduction tensor lives (a CUDA device for NCCL)."""
    import torch
    import torch.distributed as dist
    rank, world = _group()
    if world == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sharded_batch_solve(As, bs, params, solve_fn=None):
    """Solve this rank's share of the systems and gather every rank's results.

    As, bs: the whole batch (each rank passes the same list, its tensors on this rank's device).
    solve_fn(As, bs, params) -> (xs, infos, status): by default this package's batch_solve.
    Returns (xs, infos, owner): solutions on the CPU, their infos and the rank that solved each,
    all in input order and identical on every rank.
    """
    import torch.distributed as dist
    rank, world = _group()
    mine = shard_by_work([A.shape[0] for A in As], world)[rank]
    if solve_fn is None:
        from .gir import batch_solve as solve_fn
    if mine:
        xs, infos, _ = solve_fn([As[i] for i in mine], [bs[i] for i in mine], params)
    else:
        xs, infos = [], []
    local = [(i, x.detach().cpu(), info, rank) for i, x, info in zip(mine, xs, infos)]
    if world > 1:
        parts = [None] * world
        dist.all_gather_object(parts, local)
        flat = [t for part in parts for t in part]
    else:
        flat = local
    flat.sort(key=lambda t: t[0])
    if [t[0] for t in flat] != list(range(len(As))):
        raise RuntimeError("sharded batch: a system was lost or solved twice")
    return [t[1] for t in flat], [t[2] for t in flat], [t[3] for t in flat]
