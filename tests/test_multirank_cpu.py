"""Multi-rank paths on CPU ranks (gloo): the two ways the DUWP step spreads over several GPUs.

- Batch / serving (instances are independent): whole instances are placed on ranks by their
  device-memory footprint; no data moves between ranks.  Each rank runs its share through the
  oracle and the union of the ranks' results equals the whole job run in one process.
- One large instance: its cells are split into contiguous ranges, one per rank.  Every step each
  rank sends the states of its edge cells (a two-cell halo) and the particles that crossed into
  another rank's range; the split run equals the unsplit one bit for bit (world sizes 2 and 3).
Also the benchmark's host logic: whole-job throughput over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _spawn(target, world, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda x: x[0])


def _init(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)


# ------------------------------------------------------------------ benchmark host logic
def _bench_worker(rank, world, port, q):
    _init(rank, world, port)
    import torch
    import bench
    plist, cfg = bench.workload("batch64", rank, world)
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
    import bench
    out = _spawn(_bench_worker, 2)
    for rank, tmax, usum, gathered, n in out:
        assert tmax == 2.0 and usum == 21.0
        # the job is two copies of the 64-instance batch (independent seeds), each instance on one rank
        allseeds = gathered[0] + gathered[1]
        assert len(allseeds) == 128 and len(set(allseeds)) == 128
        assert bench.aggregate([10.0, 11.0], [1.0, 2.0]) == pytest.approx(usum / tmax)
    assert out[0][4] + out[1][4] == 128


def test_shard_covers_every_item_once():
    import bench
    for n in (1, 7, 64):
        for world in (1, 2, 3, 8):
            items = sorted(i for r in range(world) for i in bench.shard(n, r, world))
            assert items == list(range(n))


# ------------------------------------------------------------------ whole instances by footprint
def test_placement_covers_every_instance_once_and_balances():
    from paper_2305_12071_gb300 import placement as PL
    from paper_2305_12071_gb300 import workloads as W
    ps = W.config3_batch(64)
    for world in (1, 2, 3, 4, 8):
        a = PL.assign(ps, world)
        assert sorted(i for x in a for i in x) == list(range(64))
        loads = [sum(PL.footprint_bytes(ps[i]) for i in x) for x in a]
        # list scheduling: the loads differ by at most one instance's footprint
        assert max(loads) - min(loads) <= max(PL.footprint_bytes(p) for p in ps)
    # the footprint follows the particle count: twice the particles per cell, about twice the bytes
    p = W.shock(3.0, n_cells=200, ppc_ref=100.0, precision="fp32")
    f1, f2 = PL.footprint_bytes(p), PL.footprint_bytes(dict(p, ppc_ref=200.0))
    assert 1.9 < f2 / f1 < 2.0


def _small_batch():
    from paper_2305_12071_gb300 import workloads as W
    return W.config3_batch(6, precision="fp64", cells_range=(12, 40), ppc_range=(20, 60))


def _placed_worker(rank, world, port, q):
    _init(rank, world, port)
    import oracle as O
    from paper_2305_12071_gb300 import placement as PL
    ps = _small_batch()
    mine = PL.assign(ps, world)[rank]
    res = {}
    for i in mine:
        o = O.Oracle(ps[i])
        o.step(3)
        res[i] = (o.psi(), o.num_particles(), o.counters()["nacc"])
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    q.put((rank, gathered))
    dist.destroy_process_group()


def test_two_ranks_run_their_instances_like_one_process(oracle_mod):
    out = _spawn(_placed_worker, 2)
    merged = {}
    for part in out[0][1]:
        assert set(part).isdisjoint(merged)
        merged.update(part)
    ps = _small_batch()
    assert sorted(merged) == list(range(len(ps)))
    for i, p in enumerate(ps):
        o = oracle_mod.Oracle(p)
        o.step(3)
        psi, n, nacc = merged[i]
        assert np.array_equal(psi, o.psi()) and n == o.num_particles()
        assert np.array_equal(nacc, o.counters()["nacc"])


# ------------------------------------------------------------------ one instance over several ranks
def _split_cases():
    from paper_2305_12071_gb300 import workloads as W
    return {
        "sod_wave_fp64": W.sod(n_cells=48, Kn=3e-4, ppc_ref=50, precision="fp64", seed=7),
        "shock_fp32": W.shock(3.0, n_cells=36, ppc_ref=40, precision="fp32", seed=2),
        "periodic_vanleer_ce": W.uniform(n_cells=30, Kn=1e-3, ppc_ref=30, state=(1.0, 0.5, 0.0, 0.0, 1.0),
                                         dt=4e-3, x_max=1.0, recon_mode="vanleer", resample_mode="ce"),
    }


def _split_worker(rank, world, port, q, name, steps):
    _init(rank, world, port)
    import oracle as O
    p = _split_cases()[name]
    C = int(p["n_cells"])
    ranges = O.split_ranges(C, world)
    c0, c1 = ranges[rank]
    me = O.Oracle(p)
    me.set_range(c0, c1)
    periodic = p.get("bc_left") == "periodic"
    for _ in range(steps):
        # halo: the owned states of every rank, then the two cells beyond each end of my range
        owned = [None] * world
        dist.all_gather_object(owned, me.psi()[c0:c1])
        full = np.concatenate(owned)
        view = np.zeros((C, 5))
        view[c0:c1] = full[c0:c1]
        for c in O.halo_cells(C, c0, c1, periodic):
            view[c] = full[c]
        me.set_psi(view)
        me.first_half()
        # particles that crossed into another rank's range
        boxes = [None] * world
        dist.all_gather_object(boxes, me.outbox())
        lo, hi = O.route(boxes, ranges, rank)
        me.second_half(lo, hi)
    res = {"psi": me.psi()[c0:c1], "parts": me.particles(), "cmax": me.cmax()[c0:c1],
           "counters": {k: v[c0:c1] for k, v in me.counters().items()}}
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    q.put((rank, gathered))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name", ["sod_wave_fp64", "shock_fp32", "periodic_vanleer_ce"])
def test_domain_split_over_ranks_is_bit_identical(oracle_mod, world, name):
    steps = 12
    out = _spawn(_split_worker, world, name, steps)
    parts = out[0][1]
    o = oracle_mod.Oracle(_split_cases()[name])
    o.step(steps)
    assert np.array_equal(np.concatenate([r["psi"] for r in parts]), o.psi())
    assert np.array_equal(np.concatenate([r["cmax"] for r in parts]), o.cmax())
    ref = o.particles()
    for k in ref:
        assert np.array_equal(np.concatenate([r["parts"][k] for r in parts]), ref[k]), k
    for k, v in o.counters().items():
        assert np.array_equal(np.concatenate([r["counters"][k] for r in parts]), v), k
