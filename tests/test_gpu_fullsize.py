"""Parity at the full size of the benchmark: the 64-instance FP32 shock batch (1.28e8 particles), in
the launch configuration bench.py times (one CUDA graph per step, the free cells streaming beside
the collision kernel, 128 threads per streaming block at 64 registers), checked on sampled outputs
the oracle computes element by element (the instances small enough for the host in seconds) and
on properties that hold at any size for every instance."""
import numpy as np
import pytest

import bench
import oracle as O
from parity_util import compare_counters, compare_fields, compare_particles, solver

pytestmark = pytest.mark.gpu

REL32 = 1e-5
REL64 = 1e-9


def test_full_batch_sampled_instances_and_invariants():
    plist, _ = bench.workload("batch64", 0)
    g = solver(plist)
    g.set_launch(128, 1)
    steps = 3
    g.step(steps)
    # sampled outputs: the two smallest instances of the batch, each against the oracle
    size = [p["n_cells"] * p["ppc_ref"] for p in plist]
    for b in sorted(range(len(plist)), key=lambda i: size[i])[:2]:
        o = O.Oracle(plist[b])
        o.step(steps)
        what = f"instance {b} of the full batch"
        compare_particles(g.particles(b), o.particles(), REL32, what)
        compare_fields(g.fields(b)[0], o.psi(), REL64, what)
        compare_counters(g.counters(b), o.counters(), what)
    # every instance: a usable state, consistent counters, the steps taken, and the full particle load
    total = 0
    for b in range(len(plist)):
        n = g.num_particles(b)
        total += n
        assert n > 0, b
        f = g.fields(b)[0]
        assert np.all(np.isfinite(f)) and np.all(f[:, 0] > 0), b
        c = g.counters(b)
        assert np.all(c["nacc"] >= 0) and np.all(c["ncand"] >= c["nacc"]), b
        assert np.all(c["nabs"] == 0) and np.all(c["nnew"] >= 0), b     # P = 0 everywhere: no absorption
        assert g.info(b)["steps_done"] == steps, b
    assert total > 1.0e8
    g.close()


def test_mach8_single_instance_invariants():
    # the 1e8-particle Mach-8 shock (1e5 cells): too large for the oracle, so properties that hold at
    # any size -- a usable state everywhere, the counters consistent, the far fields at the
    # Rankine-Hugoniot states the instance starts from, the particle load of about 1e8
    from paper_2305_12071_gb300 import workloads as W
    plist, _ = bench.workload("mach8", 0)
    p = plist[0]
    g = solver(plist)
    g.set_launch(128, 1)
    g.step(3)
    f = g.fields(0)[0]
    assert np.all(np.isfinite(f)) and np.all(f[:, 0] > 0)
    c = g.counters(0)
    assert np.all(c["ncand"] >= c["nacc"]) and np.all(c["nacc"] >= 0) and np.all(c["nabs"] == 0)
    m = g.moments(0)
    r2, _, t2 = W.rankine_hugoniot(8.0)
    up, down = m["rho"][:1000].mean(), m["rho"][-1000:].mean()
    assert abs(up / p["left"][0] - 1.0) < 0.01 and abs(down / (p["left"][0] * r2) - 1.0) < 0.01, (up, down)
    assert abs(m["T"][-1000:].mean() / (p["left"][4] * t2) - 1.0) < 0.01
    assert 0.9e8 < g.num_particles(0) < 1.2e8
    g.close()
