"""Pins of the oracle's normal stress Pi = S_xx and heat flux Q = Q_x (Eq. gkt_moment1) against
what the definitions fix: hand-built particle sets with closed-form central moments (a planted
dropped -rho_p R T term, a non-central moment or a wrong power fails them), a pure-wave profile
whose central difference is exact (the NS stress and Fourier heat flux of the wave), Galilean
invariance, and the sampling bounds of a Maxwellian gas."""
import math

import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W


def _psi_of(n_cells, cell, u, v, w, mp_over_dx):
    """Total state of each cell equal to its particles' moments (so the wave is empty)."""
    psi = np.zeros((n_cells, 5))
    for i in range(n_cells):
        m = cell == i
        psi[i] = mp_over_dx * np.array([m.sum(), u[m].sum(), v[m].sum(), w[m].sum(),
                                        0.5 * (u[m] ** 2 + v[m] ** 2 + w[m] ** 2).sum()])
    return psi


def _set(o, cell, u, v, w, n_cells, mp_over_dx):
    xl = np.full(len(cell), 0.5)
    o.set_particles(cell, xl, u, v, w)
    o.set_psi(_psi_of(n_cells, cell, u, v, w, mp_over_dx))


def test_hand_built_central_moments(oracle_mod):
    # three identical cells (no gradient, so no NS part), each with the peculiar velocities below
    # about U = (0.3, -0.1, 0.2): Pi = (m/dx) (sum cx^2 - sum |c|^2 / 3), Q = (m/dx) sum cx |c|^2 / 2
    a, b = 0.7, 0.4
    c = np.array([[2 * a, b, 0.0], [-a, -b, 0.5 * b], [-a, 0.0, -0.5 * b]])
    U = np.array([0.3, -0.1, 0.2])
    C = 3
    o = oracle_mod.Oracle(W.uniform(n_cells=C, bc="periodic", ppc_ref=50, precision="fp64"))
    k = o.consts()
    mpdx = k["mp"] / k["dx"]
    cell = np.repeat(np.arange(C, dtype=np.int32), len(c))
    xi = np.tile(c + U, (C, 1))
    _set(o, cell, xi[:, 0], xi[:, 1], xi[:, 2], C, mpdx)
    r = o.stress_heat()
    s_cx2 = (c[:, 0] ** 2).sum()
    s_c2 = (c ** 2).sum()
    pi_exact = mpdx * (s_cx2 - s_c2 / 3.0)
    q_exact = mpdx * (c[:, 0] * 0.5 * (c ** 2).sum(axis=1)).sum()
    assert pi_exact != 0 and q_exact != 0
    np.testing.assert_allclose(r["Pi"], pi_exact, rtol=1e-13)
    np.testing.assert_allclose(r["Q"], q_exact, rtol=1e-13)


def test_isotropic_symmetric_set_has_no_stress_or_heat_flux(oracle_mod):
    # +-a along each axis: isotropic (Pi = 0) and odd moments vanish (Q = 0)
    a = 0.9
    c = np.array([[a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0], [0, 0, a], [0, 0, -a]])
    C = 2
    o = oracle_mod.Oracle(W.uniform(n_cells=C, bc="periodic", ppc_ref=50, precision="fp64"))
    k = o.consts()
    mpdx = k["mp"] / k["dx"]
    cell = np.repeat(np.arange(C, dtype=np.int32), len(c))
    xi = np.tile(c + np.array([1.5, 0.0, 0.0]), (C, 1))
    _set(o, cell, xi[:, 0], xi[:, 1], xi[:, 2], C, mpdx)
    r = o.stress_heat()
    scale = mpdx * len(c) * a * a
    assert np.all(np.abs(r["Pi"]) < 1e-13 * scale)
    assert np.all(np.abs(r["Q"]) < 1e-13 * scale * a)


@pytest.mark.parametrize("eps_mode", ["eps1", "eps0"])
def test_pure_wave_is_the_ns_stress_and_fourier_flux(oracle_mod, eps_mode):
    # no particles: Pi = sigma_xx = -(4/3) mu_e dU/dx, Q = q_x = -(5/2) R mu_e / Pr dT/dx with
    # mu_e = eps(dt/tau) mu(T), central differences of linear profiles (exact)
    C = 12
    p = W.uniform(n_cells=C, bc="specular", ppc_ref=50, precision="fp64", Kn=0.05, eps_mode=eps_mode,
                  dt=0.004, x_max=1.0)
    o = oracle_mod.Oracle(p)
    k = o.consts()
    dx = k["dx"]
    o.set_particles(np.zeros(0, np.int32), *(np.zeros(0) for _ in range(4)))
    x = (np.arange(C) + 0.5) * dx
    rho = np.full(C, 1.3)
    U = 0.2 + 0.75 * x
    T = 1.1 + 0.6 * x
    psi = np.stack([rho, rho * U, 0 * x, 0 * x, 0.5 * rho * U ** 2 + 1.5 * rho * T], axis=1)
    o.set_psi(psi)
    r = o.stress_heat()
    prim = o.prim()
    for i in range(1, C - 1):
        Ti, ri = prim["T"][i], prim["rho"][i]
        mu = k["mu_ref"] * (Ti / p["T_ref"]) ** p["omega"]
        tau = mu / (ri * Ti)
        mue = oracle_mod.eps(eps_mode, k["dt"] / tau) * mu
        dU = (prim["u"][i + 1] - prim["u"][i - 1]) / (2 * dx)
        dT = (prim["T"][i + 1] - prim["T"][i - 1]) / (2 * dx)
        assert dU == pytest.approx(0.75, rel=1e-12) and dT == pytest.approx(0.6, rel=1e-12)
        assert r["Pi"][i] == pytest.approx(-(4.0 / 3.0) * mue * dU, rel=1e-12)
        assert r["Q"][i] == pytest.approx(-2.5 * mue / p["Pr"] * dT, rel=1e-12)


def test_galilean_invariance(oracle_mod):
    rng = np.random.default_rng(17)
    C = 4
    o = oracle_mod.Oracle(W.uniform(n_cells=C, bc="periodic", ppc_ref=50, precision="fp64"))
    k = o.consts()
    mpdx = k["mp"] / k["dx"]
    n = 300
    cell = np.repeat(np.arange(C, dtype=np.int32), n)
    u, v, w = (rng.gamma(2.0, 0.5, C * n) - 1.0 for _ in range(3))   # skewed: Q != 0
    _set(o, cell, u, v, w, C, mpdx)
    r0 = o.stress_heat()
    _set(o, cell, u + 3.0, v - 1.0, w + 0.5, C, mpdx)
    r1 = o.stress_heat()
    scale = mpdx * n
    np.testing.assert_allclose(r1["Pi"], r0["Pi"], atol=1e-11 * scale)
    np.testing.assert_allclose(r1["Q"], r0["Q"], atol=1e-11 * scale)
    assert np.all(np.abs(r0["Q"]) > 1e-3 * scale)


def test_maxwellian_sample_within_sampling_bounds(oracle_mod):
    # N Maxwellian particles at RT = 1.7: Pi and Q vanish in expectation; standard deviations
    # (m/dx) sqrt(2N) RT for sum cx^2 - rho_p R T (an upper bound) and (m/dx) sqrt(35 N / 4) RT^1.5
    # for sum cx |c|^2 / 2 (E[cx^2 |c|^4] = 35 (RT)^3)
    rng = np.random.default_rng(5)
    N, RT = 200_000, 1.7
    o = oracle_mod.Oracle(W.uniform(n_cells=1, bc="periodic", ppc_ref=50, precision="fp64"))
    k = o.consts()
    mpdx = k["mp"] / k["dx"]
    xi = rng.normal(0.0, math.sqrt(RT), (N, 3)) + np.array([0.4, 0.0, -0.3])
    _set(o, np.zeros(N, np.int32), xi[:, 0], xi[:, 1], xi[:, 2], 1, mpdx)
    r = o.stress_heat()
    assert abs(r["Pi"][0]) < 5 * mpdx * math.sqrt(2 * N) * RT
    assert abs(r["Q"][0]) < 5 * mpdx * math.sqrt(35 * N / 4) * RT ** 1.5
    # and the scale is right: the particle pressure itself is (m/dx) N RT to sampling accuracy
    assert mpdx * (((xi - xi.mean(axis=0)) ** 2).sum() / 3) == pytest.approx(mpdx * N * RT, rel=0.02)
