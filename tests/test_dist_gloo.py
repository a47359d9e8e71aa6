"""Multi-process host logic with two gloo ranks on CPU: sequence sharding covers every
sequence exactly once with balanced work, and the job time / work combination takes the
maximum time and the summed work over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1512_05820_gb300.dist import combine, shard_by_work  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, work, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_by_work(work, rank, world)
    ms_local = 100.0 + 10.0 * rank            # pretend rank 1 is slower
    units_local = float(sum(1 for _ in mine))
    ms, units = combine(ms_local, units_local)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    q.put((rank, mine, ms, units, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_combination():
    work = [float(w) for w in [5, 1, 9, 3, 3, 7, 2, 8, 6, 4, 1, 1]]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, work, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    all_idx = sorted(i for _, mine, _, _, _ in res for i in mine)
    assert all_idx == list(range(len(work)))            # disjoint cover
    loads = [sum(work[i] for i in mine) for _, mine, _, _, _ in res]
    assert abs(loads[0] - loads[1]) <= max(work)        # balanced within one item
    for _, mine, ms, units, gathered in res:
        assert ms == 110.0 and units == len(work)       # max time, summed work
        assert gathered == [r[1] for r in res]          # every rank computed the same plan


def test_shard_single_rank_and_errors():
    assert shard_by_work([1.0, 2.0], 0, 1) == [0, 1]
    with pytest.raises(ValueError):
        shard_by_work([1.0], 2, 2)


def test_shard_properties_many_ranks():
    """Greedy longest-processing-time plans for 3 to 8 ranks on random heavy-tailed work:
    disjoint, covering, identical for every rank's call, and no rank more than one item
    above the lightest."""
    import numpy as np
    rng = np.random.default_rng(7)
    for world in range(3, 9):
        work = [float(v) for v in rng.pareto(1.5, 40) + 0.1]
        plans = [shard_by_work(work, r, world) for r in range(world)]
        assert sorted(i for p in plans for i in p) == list(range(len(work)))
        assert plans == [shard_by_work(work, r, world) for r in range(world)]
        loads = [sum(work[i] for i in p) for p in plans]
        assert max(loads) - min(loads) <= max(work)
