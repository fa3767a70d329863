"""Host logic of the multi-GPU paths on CPU: the work-balanced sharding of a batch, the gather of
results, and the maximum over ranks, with world_size-2 gloo process groups (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2201_09827_gb300.shard import shard_by_work, max_over_ranks, sharded_batch_solve


def test_shard_by_work_partition_and_balance():
    rng = np.random.default_rng(3)
    sizes = rng.integers(256, 4097, size=512)       # the batch configuration's size mix
    for world in (1, 2, 3, 8):
        parts = shard_by_work(sizes, world)
        assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
        loads = [sum(float(sizes[i]) ** 3 for i in p) for p in parts]
        # longest-processing-time: the spread is at most the largest single job
        assert max(loads) - min(loads) <= float(sizes.max()) ** 3
        assert parts == shard_by_work(sizes, world)   # deterministic
    assert shard_by_work([], 4) == [[], [], [], []]
    assert shard_by_work([100, 100], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        shard_by_work([1], 0)


def test_single_process_defaults():
    assert max_over_ranks(3.5) == 3.5
    As = [torch.eye(3) * (i + 1) for i in range(3)]
    bs = [torch.ones(3) for _ in range(3)]
    xs, infos, owner = sharded_batch_solve(As, bs, None, solve_fn=_fake_solve)
    assert owner == [0, 0, 0]
    for i, x in enumerate(xs):
        assert torch.allclose(x, torch.ones(3) / (i + 1))


def _fake_solve(As, bs, params):
    """Stand-in for the GPU batch solve: x = b / diag(A) and an info naming the system size."""
    xs = [b / torch.diagonal(A) for A, b in zip(As, bs)]
    return xs, [{"n": A.shape[0]} for A in As], 0


def _worker(rank, world, port, sizes, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        g = torch.Generator().manual_seed(7)
        As = [torch.diag(torch.rand(n, generator=g, dtype=torch.float64) + 1.0) for n in sizes]
        bs = [torch.rand(n, generator=g, dtype=torch.float64) for n in sizes]
        xs, infos, owner = sharded_batch_solve(As, bs, None, solve_fn=_fake_solve)
        m = max_over_ranks(10.0 + rank)
        torch.save({"xs": xs, "infos": infos, "owner": owner, "max": m}, os.path.join(out_dir, f"r{rank}.pt"))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_batch_two_gloo_ranks(tmp_path):
    sizes = [17, 300, 5, 64, 129, 64, 1]
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), sizes, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [torch.load(os.path.join(tmp_path, f"r{r}.pt"), weights_only=False) for r in range(world)]
    want = shard_by_work(sizes, world)
    for r in range(world):
        assert res[r]["max"] == 11.0                 # the maximum over the ranks
        assert res[r]["owner"] == res[0]["owner"]    # every rank holds the same gathered result
        assert [i["n"] for i in res[r]["infos"]] == sizes
        for q in range(world):
            assert [i for i, o in enumerate(res[r]["owner"]) if o == q] == want[q]
    g = torch.Generator().manual_seed(7)
    As = [torch.diag(torch.rand(n, generator=g, dtype=torch.float64) + 1.0) for n in sizes]
    bs = [torch.rand(n, generator=g, dtype=torch.float64) for n in sizes]
    for x, A, b in zip(res[0]["xs"], As, bs):
        assert torch.equal(x, b / torch.diagonal(A))
