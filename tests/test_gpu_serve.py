"""Continuous-batching server: requests of different sizes, Mach and Kn arrive while others are on
the GPU, are admitted by HBM footprint as slots free up, and each result equals the same problem
solved alone (bit-identical: every request draws only from its own generator key and the per-cell
arithmetic does not depend on what else is resident)."""
import time

import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W
from parity_util import solver

pytestmark = pytest.mark.gpu


def _mix():
    reqs = []
    for i, (mach, cells, ppc) in enumerate([(1.5, 120, 80), (3.0, 200, 60), (6.0, 90, 120), (2.2, 300, 40)]):
        p = W.shock(mach, n_cells=cells, ppc_ref=ppc, precision="fp32", seed=500 + i)
        reqs.append((p, 12 + 3 * i))
    for i, (kn, cells) in enumerate([(1e-3, 150), (3e-4, 110), (0.05, 250)]):
        p = W.sod(n_cells=cells, Kn=kn, ppc_ref=70, precision="fp32", seed=600 + i)
        reqs.append((p, 9 + 4 * i))
    return reqs


def _alone(p, n):
    s = solver(p)
    s.step(n)
    m = s.moments()
    s.close()
    return m


def _serve_and_compare(reqs, max_slots, max_cells, first_wave, lanes=1, long_steps=0):
    from paper_2305_12071_gb300 import build as B
    from paper_2305_12071_gb300 import duwp
    B.build()
    srv = duwp.Server(hbm_budget_bytes=2 << 30, max_slots=max_slots, max_cells=max_cells, steps_per_launch=4,
                      precision="fp32", lanes=lanes, long_steps=long_steps)
    ids = []
    # first wave, then more requests while the first ones are running
    for p, n in reqs[:first_wave]:
        ids.append(srv.submit(p, n))
    time.sleep(0.05)
    for p, n in reqs[first_wave:]:
        ids.append(srv.submit(p, n))
    results = {}
    t0 = time.time()
    while len(results) < len(ids) and time.time() - t0 < 120:
        for rid in ids:
            if rid not in results:
                r = srv.poll(rid)
                if r is not None:
                    results[rid] = r
        time.sleep(0.002)
    assert len(results) == len(ids)
    srv.close()
    for (p, n), rid in zip(reqs, ids):
        r = results[rid]
        assert r["status"] == 0
        assert r["steps"] == n
        assert r["particle_updates"] > 0
        assert r["step_p99_ms"] >= r["step_p50_ms"] > 0
        a = _alone(p, n)
        for k in ("rho", "u", "T"):
            assert np.array_equal(r[k], a[k]), f"request {rid} field {k} differs from the solve alone"


def test_served_results_equal_alone():
    _serve_and_compare(_mix(), max_slots=3, max_cells=2048, first_wave=3)


def test_two_lanes_results_equal_alone():
    # requests of at least 15 steps take the second lane, stepped beside the first on its own stream
    reqs = _mix()
    assert any(n >= 15 for _, n in reqs) and any(n < 15 for _, n in reqs)
    _serve_and_compare(reqs, max_slots=2, max_cells=2048, first_wave=4, lanes=2, long_steps=15)


def test_served_results_equal_alone_sparse_pool():
    """A pool far larger than what is resident: the step kernels cover only the cells below the
    highest resident range (in granules of 4096 cells), which grows and shrinks as requests of a few
    thousand cells are admitted into, and retired from, ranges above and below one another."""
    reqs = []
    for i, (mach, cells, ppc, n) in enumerate([(2.0, 3000, 12, 14), (4.0, 2500, 16, 6), (1.4, 4500, 10, 10),
                                               (5.0, 800, 30, 5), (3.0, 5200, 8, 9), (2.6, 1200, 20, 7)]):
        reqs.append((W.shock(mach, n_cells=cells, ppc_ref=ppc, precision="fp32", seed=700 + i), n))
    _serve_and_compare(reqs, max_slots=3, max_cells=200_000, first_wave=3)


def test_server_rejects_oversized_and_unknown():
    from paper_2305_12071_gb300 import duwp
    srv = duwp.Server(hbm_budget_bytes=256 << 20, max_slots=2, max_cells=1024, steps_per_launch=2,
                      precision="fp32")
    big = W.shock(3.0, n_cells=5000, ppc_ref=100, precision="fp32")
    with pytest.raises(duwp.DuwpError):
        srv.submit(big, 5)
    wrong = W.shock(3.0, n_cells=50, ppc_ref=50, precision="fp64")
    with pytest.raises(duwp.DuwpError):
        srv.submit(wrong, 5)
    with pytest.raises(duwp.DuwpError):
        srv.poll(987654)
    srv.close()
    with pytest.raises(duwp.DuwpError):
        duwp.Server(hbm_budget_bytes=256 << 20, max_slots=2, max_cells=1024, lanes=3)
