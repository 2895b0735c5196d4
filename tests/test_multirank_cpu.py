"""Host logic of the N > 1 benchmark path on CPU ranks (gloo, world size 2): each rank builds its
own copy of the batch with independent seeds (weak scaling, no collective on the data path), and
the whole-job throughput is all ranks' particle-updates over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plist, cfg = bench.workload("batch64", rank)
    seeds = [p["seed"] for p in plist]
    # pretend timings: rank r took (1 + r) seconds for (10 + r) updates
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    u = torch.tensor([10.0 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    q.put((rank, float(t), float(u), gathered, len(plist)))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    for rank, tmax, usum, gathered, n in out:
        assert n == 64
        assert tmax == 2.0 and usum == 21.0
        assert set(gathered[0]).isdisjoint(gathered[1])     # independent problems per rank
        assert bench.aggregate([10.0, 11.0], [1.0, 2.0]) == pytest.approx(usum / tmax)


def test_shard_covers_every_item_once():
    import bench
    for n in (1, 7, 64):
        for world in (1, 2, 3, 8):
            items = sorted(i for r in range(world) for i in bench.shard(n, r, world))
            assert items == list(range(n))
