"""Host logic of the multi-GPU paths on CPU with two gloo ranks: every rank
derives the same instance shards (disjoint, covering, DoF-balanced), and the
timing reduction returns the maximum over ranks."""
import os

import pytest

torch = pytest.importorskip("torch")


def _worker(rank, ws, port, dofs, q):
    import torch.distributed as dist

    from paper_2306_06795_gb300 import sharding

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    shards = sharding.shard_instances(dofs, ws)
    mine = shards[rank]
    gathered = [None] * ws
    dist.all_gather_object(gathered, mine)
    t = sharding.max_over_ranks(1.0 + rank * 0.5, dist)
    dist.destroy_process_group()
    q.put((rank, shards, gathered, t))


def test_two_gloo_ranks_shard_and_reduce():
    import multiprocessing as mp

    from problems import configs

    dofs = [2 * (2 * n + 1) ** 2 + (n + 1) ** 2 for n, _, _ in configs.c5_instances()]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, dofs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, g0, t0), (_, s1, g1, t1) = res
    assert s0 == s1 and g0 == g1 == s0
    flat = sorted(i for s in s0 for i in s)
    assert flat == list(range(len(dofs)))
    loads = [sum(dofs[i] for i in s) for s in s0]
    assert abs(loads[0] - loads[1]) <= max(dofs)
    assert t0 == t1 == 1.5


def test_single_rank_fallbacks():
    from paper_2306_06795_gb300 import sharding

    assert sharding.shard_instances([5, 3, 9], 1) == [[0, 1, 2]]
    assert sharding.max_over_ranks(2.5) == 2.5
    assert sharding.shard_instances([4, 4, 4, 4], 2) == [[0, 2], [1, 3]]
