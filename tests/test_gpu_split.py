"""One instance split into cell ranges on the GPU (duwp_split_*): every step the parts exchange the
particles that crossed into each other's cells and a one-cell halo of the state, so the split run
must equal the undivided one bit for bit -- particles in the stable per-cell order, Psi_t, c_max and
the per-cell counters -- and match the oracle's host-rank emulation of the same split."""
import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W
from parity_util import solver

pytestmark = pytest.mark.gpu


def _cases():
    return {
        "shock_fp64": W.shock(3.0, n_cells=60, ppc_ref=60, precision="fp64", seed=2),
        "shock_fp32": W.shock(5.0, n_cells=90, ppc_ref=50, precision="fp32", seed=3),
        "sod_wave_fp32": W.sod(n_cells=120, Kn=3e-4, ppc_ref=80, precision="fp32", seed=4),
        "sod_wave_ce_fp64": W.sod(n_cells=80, Kn=3e-4, ppc_ref=60, precision="fp64", seed=5, resample_mode="ce"),
        "expansion_fp32": W.base(n_cells=64, left=(1, 0, 0, 0, 1), right=(0, 0, 0, 0, 1), x_split=0.5,
                                 bc_left="specular", bc_right="vacuum", ppc_ref=60, Kn=0.05, dt=0.004,
                                 precision="fp32"),
    }


def _same(a, b):
    pa, pb = a.particles(), b.particles()
    assert len(pa["cell"]) == len(pb["cell"])
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    assert np.array_equal(a.fields()[0] if hasattr(a, "n") else a.fields(), b.fields())
    assert np.array_equal(a.cmax(), b.cmax())
    ca, cb = a.counters(), b.counters()
    for k in ca:
        assert np.array_equal(ca[k], cb[k]), k


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("parts", [2, 3, 7])
def test_split_equals_undivided(name, parts):
    from paper_2305_12071_gb300 import duwp
    p = _cases()[name]
    whole = solver(p)
    split = duwp.Split(p, parts)
    for _ in range(3):
        whole.step(6)
        split.step(6)
        _same(whole, split)
    assert split.particle_updates() == whole.particle_updates()
    split.close()
    whole.close()


def test_split_matches_oracle_split(oracle_mod):
    from paper_2305_12071_gb300 import duwp
    p = _cases()["sod_wave_ce_fp64"]
    g = duwp.Split(p, 3)
    o = oracle_mod.DomainSplit(p, 3)
    g.step(10)
    o.step(10)
    gp, op = g.particles(), o.particles()
    assert np.array_equal(gp["cell"], op["cell"])
    for k in ("xl", "u", "v", "w"):
        assert np.max(np.abs(gp[k] - op[k]) / np.maximum(np.abs(op[k]), 1.0)) <= 1e-9
    assert np.array_equal(g.counters()["ncand"], o.counters()["ncand"])
    g.close()


def test_split_refuses_what_it_does_not_cover():
    from paper_2305_12071_gb300 import duwp
    with pytest.raises(duwp.DuwpError):
        duwp.Split(W.uniform(n_cells=20, Kn=1e-2, ppc_ref=20), 2)                     # periodic ends
    with pytest.raises(duwp.DuwpError):
        duwp.Split(W.sod(n_cells=40, Kn=1e-3, ppc_ref=20, recon_mode="vanleer"), 2)  # two-cell reach
