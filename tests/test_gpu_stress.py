"""Parity of the stress / heat-flux read-out (Eq. gkt_moment1) with the oracle on the same seeded
problems: the particle central moments about U_t plus the wave's NS stress and heat flux weighted
by rho_w / rho_t, per cell, after the same steps.  The two sides sum the same particle values in
different orders, so Pi and Q agree to rounding: within 1e-9 of the largest cell pressure (FP64
records; the particle state and Psi_t themselves agree to 1e-9) and 1e-5 (FP32 records over 5
steps); the time average of the accumulated states against the mean of the oracle's per-step
values."""
import numpy as np
import pytest

import oracle as O
from paper_2305_12071_gb300 import duwp
from paper_2305_12071_gb300 import workloads as W
from parity_util import solver

pytestmark = pytest.mark.gpu


def _scale(o):
    """Largest cell pressure p and p sqrt(2RT) of the oracle's state (R = 1): the error scale, as
    the field comparisons take the largest magnitude over the cells."""
    pr = o.prim()
    p = pr["rho"] * pr["T"]
    return max(p.max(), 1e-300), max((p * np.sqrt(2.0 * np.maximum(pr["T"], 0.0))).max(), 1e-300)


def _compare(g, o, rel, what, inst=0):
    a, b = g.stress_heat(inst), o.stress_heat()
    sp, sq = _scale(o)
    ep = np.abs(a["Pi"] - b["Pi"]) / sp
    eq = np.abs(a["Q"] - b["Q"]) / sq
    assert ep.max() <= rel, f"{what}: Pi rel err {ep.max():.3e} at cell {int(np.argmax(ep))}"
    assert eq.max() <= rel, f"{what}: Q rel err {eq.max():.3e} at cell {int(np.argmax(eq))}"
    return a, b


@pytest.mark.parametrize("precision,steps,rel", [("fp64", [1, 5, 20], 1e-9), ("fp32", [1, 5], 1e-5)])
def test_shock_stress_heat(precision, steps, rel):
    p = W.config1(precision)
    g, o = solver(p), O.Oracle(p)
    done = 0
    for n in steps:
        g.step(n - done)
        o.step(n - done)
        done = n
        a, b = _compare(g, o, rel, f"step {n}")
    # the shock carries a real stress and heat flux (not a comparison of zeros)
    sp, sq = _scale(o)
    assert np.abs(b["Pi"] / sp).max() > 0.05 and np.abs(b["Q"] / sq).max() > 0.02
    g.close()


@pytest.mark.parametrize("resample_mode", ["maxwell", "ce"])
def test_wave_regime_stress_heat(resample_mode):
    # P > 0: the wave holds most of the mass, its NS part dominates the dense side
    p = W.sod(n_cells=120, Kn=1e-4, ppc_ref=150, precision="fp64", seed=7, resample_mode=resample_mode)
    g, o = solver(p), O.Oracle(p)
    done = 0
    for n in (1, 3, 10):
        g.step(n - done)
        o.step(n - done)
        done = n
        _compare(g, o, 1e-9, f"step {n}")
    m = g.moments()
    assert m["wave_frac"].max() > 0.5
    g.close()


def test_time_averaged_stress_heat():
    p = W.config1("fp64")
    g, o = solver(p), O.Oracle(p)
    g.step(3)
    o.step(3)
    z = g.stress_heat(which=duwp.AVERAGED)
    assert not z["Pi"].any() and not z["Q"].any()
    acc_p, acc_q = 0.0, 0.0
    for _ in range(8):
        g.step(1)
        g.stress_heat_accumulate()
        o.step(1)
        r = o.stress_heat()
        acc_p = acc_p + r["Pi"]
        acc_q = acc_q + r["Q"]
    a = g.stress_heat(which=duwp.AVERAGED)
    sp, sq = _scale(o)
    assert (np.abs(a["Pi"] - acc_p / 8) / sp).max() <= 1e-9
    assert (np.abs(a["Q"] - acc_q / 8) / sq).max() <= 1e-9
    g.close()


def test_batch_instances_and_ragged_sizes():
    # instances of a batch read out separately, ragged sizes (1, 2 and 37 cells, an empty-ish cell)
    plist = [W.uniform(n_cells=1, ppc_ref=40, precision="fp64", seed=3),
             W.shock(2.0, n_cells=37, ppc_ref=30, precision="fp64", seed=4),
             W.uniform(n_cells=2, ppc_ref=3, precision="fp64", seed=5, state=(1.0, 0.2, 0.0, 0.0, 2.0))]
    g = solver(plist)
    orcs = [O.Oracle(q) for q in plist]
    g.step(4)
    for b, o in enumerate(orcs):
        o.step(4)
        _compare(g, o, 1e-9, f"instance {b}", inst=b)
    with pytest.raises(duwp.DuwpError):
        g.stress_heat(0, which=7)
    buf = np.zeros(64)
    ptr = buf.ctypes.data_as(duwp.C.POINTER(duwp.C.c_double))
    assert g.L.duwp_stress_heat(g.h, 3, 0, ptr, ptr, 1) == duwp.EINVAL      # no such instance
    assert g.L.duwp_stress_heat(g.h, 1, 0, ptr, ptr, 36) == duwp.EINVAL     # wrong cell count
    g.close()
