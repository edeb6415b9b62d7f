"""Host-side logic of the multi-GPU paths: independent instances are
sharded across ranks with no data-path collective (each rank solves its
own instances), and timings are combined as the maximum over ranks."""


def shard_instances(dofs, world_size):
    """Assign instances to ranks, balancing DoFs: largest first, each to the
    least-loaded rank (lowest rank on ties).  Deterministic; returns, per
    rank, the ascending list of its instance indices."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    load = [0] * world_size
    out = [[] for _ in range(world_size)]
    for i in sorted(range(len(dofs)), key=lambda k: (-dofs[k], k)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += dofs[i]
    return [sorted(o) for o in out]


def max_over_ranks(value, dist=None, device="cpu"):
    """The maximum of a per-rank float over all ranks (the value itself
    without an initialised process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
