"""Host-side logic of multi-GPU runs (one process per GPU; no collective on the data path).

Independent sequences shard across ranks; each rank solves its own share and only the
timings and counts are combined: the job time is the maximum over ranks (everyone waits
for the slowest) and the work is the sum. A single sequence does not shard (its systems
depend on each other through the snapshots), so several GPUs run independent replicas.
"""
from __future__ import annotations


def shard_by_work(work: list[float], rank: int, world: int) -> list[int]:
    """Indices of the items rank `rank` solves: greedy longest-processing-time assignment
    (items in decreasing work order, each to the least-loaded rank; ties to the lower rank),
    identical on every rank, disjoint, covering all items."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    load = [0.0] * world
    owner = [0] * len(work)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += work[i]
    return [i for i in range(len(work)) if owner[i] == rank]


def combine(ms_local: float, units_local: float, group=None) -> tuple[float, float]:
    """(max over ranks of the elapsed ms, sum over ranks of the units processed)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return ms_local, units_local
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(u.item())
