"""Pins of the oracle's second-order wave reconstruction (recon_mode = vanleer): the van Leer
limited slope is exact on linear data (the interface sees the midpoint from both sides), vanishes at
an extremum, never overshoots the neighbouring states (TVD) and leaves a uniform state alone; in a
step, the wave flux of a linear density profile at rest is the flux of the uniform midpoint state
(a dropped factor 1/2, a wrong sign or the minmod slope fail these)."""
import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W


def test_linear_data_reconstructs_the_midpoint(oracle_mod):
    base = np.array([1.0, 0.3, -0.1, 0.05, 1.2])
    d = np.array([0.07, -0.02, 0.01, 0.003, 0.05])
    Wm, W0, W1, W2 = (base + k * d for k in range(4))
    L, R = oracle_mod.recon_pair(Wm, W0, W1, W2)
    mid = 0.5 * (W0 + W1)
    np.testing.assert_allclose(L, mid, rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(R, mid, rtol=1e-14, atol=1e-16)


def test_extremum_has_zero_slope_and_harmonic_mean_otherwise(oracle_mod):
    # density peaks at W0 (zero slope there); velocity has one-sided differences 0.1 and 0.3:
    # van Leer slope 2*0.1*0.3/0.4 = 0.15 (minmod would give 0.1, the central slope 0.2)
    Wm = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    W0 = np.array([1.5, 0.1, 0.0, 0.0, 1.0])
    W1 = np.array([1.2, 0.4, 0.0, 0.0, 1.0])
    W2 = np.array([1.1, 0.9, 0.0, 0.0, 1.0])
    L, R = oracle_mod.recon_pair(Wm, W0, W1, W2)
    assert L[0] == W0[0]
    assert L[1] == pytest.approx(0.1 + 0.5 * 0.15, rel=1e-14)
    # right cell: density differences -0.3, -0.1 -> slope 2*0.03/(-0.4) = -0.15
    assert R[0] == pytest.approx(1.2 + 0.5 * 0.15, rel=1e-14)
    # velocity at the right cell: 0.3 and 0.5 -> 0.375
    assert R[1] == pytest.approx(0.4 - 0.5 * 0.375, rel=1e-14)


def test_tvd_and_uniform(oracle_mod):
    rng = np.random.default_rng(3)
    for _ in range(500):
        # monotone (per component) random sequences of four states
        steps = rng.exponential(1.0, (3, 5)) * rng.choice([-1.0, 1.0], 5)
        Wm = np.array([2.0, 0.0, 0.0, 0.0, 2.0]) + rng.normal(0, 0.1, 5)
        seq = [Wm]
        for k in range(3):
            seq.append(seq[-1] + 0.1 * steps[k])
        if min(s[0] for s in seq) <= 0 or min(s[4] for s in seq) <= 0:
            continue
        L, R = oracle_mod.recon_pair(*seq)
        lo = np.minimum(seq[1], seq[2]) - 1e-14
        hi = np.maximum(seq[1], seq[2]) + 1e-14
        assert np.all(L >= lo) and np.all(L <= hi)
        assert np.all(R >= lo) and np.all(R <= hi)
    U = np.array([0.8, 0.2, 0.0, 0.1, 1.4])
    L, R = oracle_mod.recon_pair(U, U, U, U)
    assert np.array_equal(L, U) and np.array_equal(R, U)


def test_step_flux_of_linear_density_is_the_midpoint_flux(oracle_mod):
    # all wave, U = 0, uniform T: no viscous term; the second-order interface states are the
    # midpoint state on both sides, so the flux is that uniform state's flux
    C = 16
    p = W.uniform(n_cells=C, Kn=1e-5, ppc_ref=20, state=(1, 0, 0, 0, 1), bc="specular", dt=2e-3, x_max=1.0,
                  recon_mode="vanleer")
    o = oracle_mod.Oracle(p)
    o.set_particles(np.zeros(0, np.int32), *(np.zeros(0) for _ in range(4)))
    rho = 1.0 + 0.02 * np.arange(C)
    T = 1.3
    psi = np.zeros((C, 5))
    psi[:, 0] = rho
    psi[:, 4] = 1.5 * rho * T
    o.set_psi(psi)
    o.step(1)
    F = o.last_flux()
    o1 = oracle_mod.Oracle(dict(p, recon_mode="first"))
    o1.set_particles(np.zeros(0, np.int32), *(np.zeros(0) for _ in range(4)))
    o1.set_psi(psi)
    o1.step(1)
    F1 = o1.last_flux()
    for f in range(2, C - 1):
        mid = np.array([0.5 * (rho[f - 1] + rho[f]), 0.0, 0.0, 0.0, T])
        Fm = oracle_mod.wave_flux(p, mid, mid)
        np.testing.assert_allclose(F[f], Fm, rtol=1e-12, atol=1e-14)
        # first order sees two different half-Maxwellians: a net mass flux down the gradient
        assert F1[f][0] < -1e-6 and abs(F[f][0]) < 1e-14
