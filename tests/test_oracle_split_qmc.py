"""Pins of the oracle's split_mode = qmc (Sec. 3.2: the multi-scale Boltzmann equation solved by
quantified model competition; Sec. 3.3: the flux at t = dt) against what its definitions fix:
the collision probability 1 - exp(-dt/tau) with tau = mu(T)/p in closed form and in its two
limits, the flux of a uniform state as (1 - exp(-dt/tau)) times the Euler flux, absorption
counts against Binomial(n, P), and the ordering against Eq. (p)."""
import math

import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W


def _tau(o, p, rho, T):
    k = o.consts()
    mu = k["mu_ref"] * (T / p["T_ref"]) ** p["omega"]
    return mu / (rho * p["R"] * T), k["dt"]


@pytest.mark.parametrize("Kn,state", [(1e-3, (1.0, 0.2, 0.0, 0.0, 1.0)), (0.05, (0.4, 0.0, 0.1, 0.0, 2.5)),
                                      (5.0, (1.7, -0.3, 0.0, 0.2, 0.6))])
def test_collision_probability_closed_form(oracle_mod, Kn, state):
    p = W.uniform(n_cells=4, Kn=Kn, ppc_ref=20, state=state, dt=2e-3, x_max=1.0, split_mode="qmc")
    o = oracle_mod.Oracle(p)
    pr = o.prim()
    tau, dt = _tau(o, p, state[0], state[4])
    exact = -math.expm1(-dt / tau)
    np.testing.assert_allclose(pr["P"], exact, rtol=1e-12)
    # Eq. (p) never exceeds it (1 - 1/x <= 1 - exp(-x) for every x > 0)
    q = oracle_mod.Oracle(dict(p, split_mode="p")).prim()["P"]
    assert np.all(q <= pr["P"])


def test_collision_probability_limits(oracle_mod):
    # dt << tau: P = dt/tau (1 - dt/(2 tau) + ...); dt >> tau: P -> 1 (Eq. p would give 1 - tau/dt)
    rare = W.uniform(n_cells=2, Kn=50.0, ppc_ref=20, state=(1, 0, 0, 0, 1), dt=1e-3, x_max=1.0, split_mode="qmc")
    o = oracle_mod.Oracle(rare)
    tau, dt = _tau(o, rare, 1.0, 1.0)
    x = dt / tau
    assert x < 1e-4
    assert o.prim()["P"][0] == pytest.approx(x * (1 - x / 2), rel=1e-8)
    cont = dict(rare, Kn=1e-6)
    o = oracle_mod.Oracle(cont)
    tau, dt = _tau(o, cont, 1.0, 1.0)
    assert dt / tau > 100
    assert o.prim()["P"][0] == 1.0 or 1.0 - o.prim()["P"][0] < 1e-40


@pytest.mark.parametrize("flux", ["gks_eq", "kfvs"])
@pytest.mark.parametrize("Kn", [1e-4, 0.3, 30.0])
def test_uniform_flux_weight(oracle_mod, flux, Kn):
    W5 = (0.8, 0.45, 0.1, -0.2, 1.3)
    rho, u, v, w, T = W5
    pr = rho * T
    E = 0.5 * rho * (u * u + v * v + w * w) + 1.5 * pr
    euler = np.array([rho * u, rho * u * u + pr, rho * u * v, rho * u * w, u * (E + pr)])
    p = W.base(Kn=Kn, n_cells=100, flux_mode=flux, dt=1e-3, split_mode="qmc")
    F = oracle_mod.wave_flux(p, W5, W5)
    o = oracle_mod.Oracle(W.uniform(n_cells=2, Kn=Kn, ppc_ref=20, state=W5, dt=1e-3, x_max=1.0))
    k = o.consts()
    tau = k["mu_ref"] * T ** p["omega"] / pr
    weight = -math.expm1(-k["dt"] / tau)
    # in a uniform state the interface equilibrium is the state itself (and KFVS sums to Euler)
    np.testing.assert_allclose(F, weight * euler, rtol=1e-12, atol=1e-15 * np.abs(euler).max())
    if Kn == 30.0:
        # rarefied: Eq. (p) gives no wave flux at all, the QMC weight a small positive one
        assert np.all(oracle_mod.wave_flux(dict(p, split_mode="p"), W5, W5) == 0.0)
        assert 0.0 < weight < 1e-3


def test_absorption_counts_follow_binomial(oracle_mod):
    # transition regime: P = 1 - exp(-dt/tau) per particle, absorbed ~ Binomial(n, P)
    p = W.uniform(n_cells=10, Kn=2e-3, ppc_ref=3000, state=(1.0, 0.0, 0.0, 0.0, 1.0), dt=2e-3, x_max=1.0,
                  split_mode="qmc")
    o = oracle_mod.Oracle(p)
    o.step(2)
    n_before = o.num_particles()
    P = o.prim()["P"].mean()
    o.step(1)
    nabs = o.counters()["nabs"].sum()
    assert 0.2 < P < 0.9
    assert abs(nabs - P * n_before) < 5 * math.sqrt(n_before * P * (1 - P))
