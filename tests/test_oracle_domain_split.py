"""The oracle's domain decomposition (one instance's cells split into contiguous ranges, each part
owning its range: the host-rank emulation of running one large instance over several GPUs) against
the undivided run, bit for bit: every boundary kind, both record precisions, the second-order
reconstruction (two-cell halo) and the NS-corrected re-sampling, down to one cell per part (far
movers then cross several parts).  A halo one cell too thin for the reconstruction, or the arriving
particles merged in the wrong order, must break the equality."""
import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W


def _cases():
    return {
        "sod_wave": W.sod(n_cells=40, Kn=3e-4, ppc_ref=50, precision="fp64", seed=3),
        "shock_fp32": W.shock(3.0, n_cells=32, ppc_ref=40, precision="fp32", seed=4),
        "periodic": W.uniform(n_cells=24, Kn=3e-3, ppc_ref=40, state=(1.0, 0.4, 0.0, 0.0, 1.0), dt=2e-3, x_max=1.0),
        "vanleer_ce": W.sod(n_cells=36, Kn=3e-4, ppc_ref=40, precision="fp64", seed=5, recon_mode="vanleer",
                            resample_mode="ce"),
        "qmc": W.shock(2.0, n_cells=30, ppc_ref=40, precision="fp64", split_mode="qmc"),
        "vacuum": W.base(n_cells=30, left=(1, 0, 0, 0, 1), right=(0, 0, 0, 0, 1), x_split=0.5, bc_left="specular",
                         bc_right="vacuum", ppc_ref=40, Kn=1.0, dt=0.01),
    }


def _same(a, b):
    pa, pb = a.particles(), b.particles()
    if len(pa["u"]) != len(pb["u"]):
        return False
    ok = all(np.array_equal(pa[k], pb[k]) for k in pa) and np.array_equal(a.psi(), b.psi())
    ok = ok and np.array_equal(a.cmax(), b.cmax())
    ca, cb = a.counters(), b.counters()
    return ok and all(np.array_equal(ca[k], cb[k]) for k in ca)


@pytest.mark.parametrize("name", list(_cases()))
def test_split_equals_undivided(oracle_mod, name):
    p = _cases()[name]
    for parts in (2, 3, int(p["n_cells"])):
        a, b = oracle_mod.Oracle(p), oracle_mod.DomainSplit(p, parts)
        a.step(10)
        b.step(10)
        assert _same(a, b), (name, parts)


def test_split_ranges_and_halo(oracle_mod):
    assert oracle_mod.split_ranges(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert sorted(oracle_mod.halo_cells(10, 3, 6, False)) == [1, 2, 6, 7]
    assert sorted(oracle_mod.halo_cells(10, 0, 3, False)) == [3, 4]
    assert sorted(oracle_mod.halo_cells(10, 0, 3, True)) == [3, 4, 8, 9]


def test_planted_mistakes_break_the_split(oracle_mod, monkeypatch):
    p = _cases()["vanleer_ce"]
    a = oracle_mod.Oracle(p)
    a.step(6)
    # a one-cell halo misses the second neighbour the reconstruction reads
    real_halo = oracle_mod.halo_cells
    monkeypatch.setattr(oracle_mod, "halo_cells", lambda C, c0, c1, per, width=2: real_halo(C, c0, c1, per, 1))
    b = oracle_mod.DomainSplit(p, 3)
    b.step(6)
    assert not _same(a, b)
    monkeypatch.setattr(oracle_mod, "halo_cells", real_halo)
    # particles from higher parts merged before those from lower parts
    real_route = oracle_mod.route
    monkeypatch.setattr(oracle_mod, "route", lambda boxes, ranges, me: real_route(boxes, ranges, me)[::-1])
    q = _cases()["shock_fp32"]
    a = oracle_mod.Oracle(q)
    a.step(6)
    b = oracle_mod.DomainSplit(q, 4)
    b.step(6)
    assert not _same(a, b)
    # the particles from lower parts in reverse order
    monkeypatch.setattr(oracle_mod, "route", lambda boxes, ranges, me: _swap_inside(real_route(boxes, ranges, me)))
    b = oracle_mod.DomainSplit(q, 4)
    b.step(6)
    assert not _same(a, b)


def _swap_inside(lohi):
    """Reverse the order of the particles arriving from lower parts (still a valid merge input)."""
    lo, hi = lohi
    return {k: v[::-1].copy() for k, v in lo.items()}, hi
