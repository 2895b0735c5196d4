"""Pins of the oracle's closed-form pieces, each checked by an independent route:
the mean-free-path constant against the VHS viscosity/mean-free-path relations, the
reference relative speed against an equilibrium quadrature, the NTC candidate count
against the dimensional form of Appendix A, the viscosity-correction factors against
quadratures of the integral solution (Sec. 3.3), the half-Maxwellian moments against
quadrature, and the interface flux against the Euler flux and its symmetries."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2305_12071_gb300 import workloads as W


@pytest.mark.parametrize("omega", [0.5, 0.68, 0.74, 0.81, 1.0])
def test_beta_matches_vhs_viscosity_and_hard_sphere_mean_free_path(oracle_mod, omega):
    # Physical units, argon-like numbers (any positive values work).
    k, m, d, n, T = 1.380649e-23, 6.63e-26, 4.17e-10, 1.3e20, 273.0
    R = k / m
    p = n * k * T
    # VHS viscosity at the reference temperature (first Chapman-Enskog approximation)
    mu = 15.0 * math.sqrt(math.pi * m * k * T) / (2.0 * (5 - 2 * omega) * (7 - 2 * omega) * math.pi * d * d)
    lam_hs = 1.0 / (math.sqrt(2.0) * math.pi * d * d * n)      # second form of Eq. (lambda)
    b = oracle_mod.beta(omega, 1.0)
    lam_first = (1.0 / b) * (mu / p) * math.sqrt(R * T / (2 * math.pi))  # first form
    assert lam_first == pytest.approx(lam_hs, rel=1e-12)


@pytest.mark.parametrize("omega", [0.6, 0.68, 0.81, 0.95])
def test_c_ref_makes_equilibrium_cross_section_average_hard_sphere(oracle_mod, omega):
    # Relative speeds of an equilibrium gas at T_ref (reduced mass m/2): density
    # (4/sqrt(pi)) c^2 a^{-3/2} exp(-c^2/a) with a = 2kT/m_r = 4 R T_ref.
    R, Tref = 1.0, 1.0
    a = 4 * R * Tref
    f = lambda c: 4 / math.sqrt(math.pi) * c * c / a**1.5 * math.exp(-c * c / a)
    cr = oracle_mod.c_ref(omega, R, Tref)
    ups = omega - 0.5
    sig_c = integrate.quad(lambda c: (c / cr) ** (-2 * ups) * c * f(c), 0, np.inf)[0]
    c_mean = integrate.quad(lambda c: c * f(c), 0, np.inf)[0]
    assert sig_c == pytest.approx(c_mean, rel=1e-9)


@pytest.mark.parametrize("omega,N,cmax", [(0.81, 350, 11.0), (0.5, 40, 6.0), (1.0, 1000, 3.0), (0.68, 2, 20.0)])
def test_ntc_count_equals_dimensional_form(oracle_mod, omega, N, cmax):
    prm = W.base(omega=omega, Kn=0.37, L_ref=2.0, x_min=0.0, x_max=3.0, n_cells=6, ppc_ref=123.0, dt=0.011)
    lam_ref = 0.37 * 2.0
    Vc = 0.5
    Nref = 123.0
    FN = 3.0e11                                   # real molecules per simulated particle
    n_ref = FN * Nref / Vc
    d2 = 1.0 / (math.sqrt(2) * math.pi * lam_ref * n_ref)
    cr = oracle_mod.c_ref(omega, 1.0, 1.0)
    ups = omega - 0.5
    sigma_max = math.pi * d2 * (cmax / cr) ** (-2 * ups)
    direct = 0.5 * N * (N - 1) * FN * sigma_max * cmax * 0.011 / Vc
    got = oracle_mod.ntc_nsel(prm, N / Nref, float(N), cmax)
    assert got == pytest.approx(direct, rel=1e-12)


@pytest.mark.parametrize("x", [1e-3, 0.1, 0.7, 2.0, 9.0, 40.0])
def test_eps1_from_integral_solution_at_dt(oracle_mod, x):
    # Coefficient of the spatial derivative in the integral solution at t = dt over the
    # coefficient of the equilibrium term, divided by tau (Sec. 3.3): eps1.
    tau = 1.0
    dt = x * tau
    num = integrate.quad(lambda s: s * math.exp(-s / tau), 0, dt, epsabs=0, epsrel=1e-13)[0]
    den = tau * integrate.quad(lambda s: math.exp(-s / tau), 0, dt, epsabs=0, epsrel=1e-13)[0]
    assert oracle_mod.eps("eps1", x) == pytest.approx(num / den, rel=1e-9)


@pytest.mark.parametrize("x", [0.05, 0.5, 1.0, 3.0, 12.0])
def test_eps_avg_from_time_averaged_flux_coefficients(oracle_mod, x):
    # delta_1, delta_2 as time integrals of the integral solution (Eqs. flux, expansion):
    # delta_1 = int_0^dt (1 - e^{-t/tau}) dt,
    # delta_2 = -(1/tau) int_0^dt int_0^t (t - s) e^{(s-t)/tau} ds dt;  eps = -delta_2/(tau delta_1).
    tau = 1.0
    dt = x * tau
    d1 = integrate.quad(lambda t: 1 - math.exp(-t / tau), 0, dt, epsrel=1e-13)[0]
    d2 = -(1 / tau) * integrate.dblquad(lambda s, t: (t - s) * math.exp((s - t) / tau), 0, dt,
                                        lambda t: 0.0, lambda t: t, epsabs=1e-15, epsrel=1e-12)[0]
    assert oracle_mod.eps("eps_avg", x) == pytest.approx(-d2 / (tau * d1), rel=1e-7)


def test_eps_limits_and_second_order_form(oracle_mod):
    for mode in ("eps1", "eps_avg", "eps12"):
        assert oracle_mod.eps(mode, 800.0) == pytest.approx(1.0, abs=5e-3)
    assert oracle_mod.eps("eps1", 1e6) == 1.0
    for x in (1e-4, 1e-3):
        assert oracle_mod.eps("eps1", x) == pytest.approx(x / 2 - x * x / 12, rel=1e-6)
        assert oracle_mod.eps("eps_avg", x) == pytest.approx(x / 3, rel=2e-3)
    assert oracle_mod.eps("eps0", 0.3) == 1.0
    # eps12: eps1 with e^{-x} replaced by 1/(1 + x + x^2/2)
    for x in (0.01, 0.3, 2.0, 7.0):
        e = 1.0 / (1 + x + x * x / 2)
        assert oracle_mod.eps("eps12", x) == pytest.approx(1 - x * e / (1 - e), rel=1e-12)


@pytest.mark.parametrize("U,T", [(0.0, 1.0), (0.7, 2.0), (-3.1, 0.4), (5.0, 1.0)])
def test_half_maxwellian_moments_by_quadrature(oracle_mod, U, T):
    lam = 1.0 / (2.0 * T)
    g = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
    Mp, Mm = oracle_mod.half_moments(U, lam)
    for n in range(4):
        qp = integrate.quad(lambda u: u**n * g(u), 0, np.inf, epsabs=1e-14, epsrel=1e-12)[0]
        qm = integrate.quad(lambda u: u**n * g(u), -np.inf, 0, epsabs=1e-14, epsrel=1e-12)[0]
        assert Mp[n] == pytest.approx(qp, rel=1e-9, abs=1e-13)
        assert Mm[n] == pytest.approx(qm, rel=1e-9, abs=1e-13)


def _euler_flux(W5):
    rho, u, v, w, T = W5
    p = rho * T
    E = 0.5 * rho * (u * u + v * v + w * w) + 1.5 * p
    return np.array([rho * u, rho * u * u + p, rho * u * v, rho * u * w, u * (E + p)])


@pytest.mark.parametrize("flux", ["gks_eq", "kfvs"])
@pytest.mark.parametrize("W5", [(1.0, 0.3, 0.1, -0.2, 1.0), (0.125, -1.2, 0.0, 0.0, 0.8), (3.0, 1.29, 0.0, 0.0, 3.67)])
def test_flux_of_uniform_state_is_weighted_euler_flux(oracle_mod, flux, W5):
    cont = W.base(Kn=1e-8, n_cells=100, flux_mode=flux, dt=1e-3)
    F = oracle_mod.wave_flux(cont, W5, W5)
    E = _euler_flux(W5)
    nz = np.abs(E) > 0
    assert np.all(F[~nz] == 0.0)
    ratio = F[nz] / E[nz]
    # one common weight P_f close to 1 in the continuum, applied to all components
    assert np.all(np.abs(ratio - ratio[0]) < 1e-12)
    assert 0.99 < ratio[0] <= 1.0
    rare = W.base(Kn=10.0, n_cells=100, flux_mode=flux, dt=1e-3)
    assert np.all(oracle_mod.wave_flux(rare, W5, W5) == 0.0)


@pytest.mark.parametrize("flux", ["gks_eq", "kfvs"])
def test_flux_mirror_symmetry(oracle_mod, flux):
    prm = W.base(Kn=1e-6, n_cells=50, flux_mode=flux, dt=2e-3)
    L = (1.0, 0.4, 0.2, -0.1, 1.3)
    R = (0.3, -0.2, 0.05, 0.3, 0.7)
    F = oracle_mod.wave_flux(prm, L, R)
    mir = lambda s: (s[0], -s[1], s[2], s[3], s[4])
    G = oracle_mod.wave_flux(prm, mir(R), mir(L))
    assert F[0] == pytest.approx(-G[0], rel=1e-12)
    assert F[1] == pytest.approx(G[1], rel=1e-12)
    assert F[2] == pytest.approx(-G[2], rel=1e-12)
    assert F[3] == pytest.approx(-G[3], rel=1e-12)
    assert F[4] == pytest.approx(-G[4], rel=1e-12)


def test_viscous_terms_newtonian_stress_and_monatomic_conductivity(oracle_mod):
    # Small gradients around a state at rest: the viscous parts of the flux are
    # -(4/3) mu_e dU/dx (normal), -mu_e dV/dx (shear) and -kappa_e dT/dx with
    # kappa = (15/4) R mu for a monatomic gas at Pr = 2/3.
    prm = W.base(Kn=1e-3, n_cells=100, x_min=0.0, x_max=1.0, dt=2e-3)
    dx = 0.01
    h = 1e-7
    base = (1.0, 0.0, 0.0, 0.0, 1.0)

    def visc(L, R):
        return oracle_mod.wave_flux(prm, L, R, True) - oracle_mod.wave_flux(prm, L, R, False)

    dn = visc((1.0, -h, 0, 0, 1.0), (1.0, h, 0, 0, 1.0))        # dU/dx = 2h/dx
    ds = visc((1.0, 0, -h, 0, 1.0), (1.0, 0, h, 0, 1.0))        # dV/dx = 2h/dx
    dT = visc((1.0 + h, 0, 0, 0, 1.0 - h), (1.0 - h, 0, 0, 0, 1.0 + h))  # dT/dx = 2h/dx, p ~ const
    mu_e_shear = -ds[2] / (2 * h / dx)
    mu_e_norm = -dn[1] / (2 * h / dx) * 3.0 / 4.0
    kap = -dT[4] / (2 * h / dx)
    assert mu_e_shear > 0
    assert mu_e_norm == pytest.approx(mu_e_shear, rel=1e-5)
    assert kap / mu_e_shear == pytest.approx(15.0 / 4.0, rel=1e-5)
    # shear stress does no work at rest, the normal stress term carries U0 = O(h)
    assert abs(ds[4]) < 1e-12
    assert base[1] == 0.0
