"""Closed-form pins of Eq. (p) (the fraction P of a cell's particles absorbed into the wave) and of
the weight P_f of the wave flux (Sec. 3.3, with the reading that the flux is weighted like Eq. (p)
at the interface state), both checked against values the test builds by routes of its own:

- tau = mu(T) / p with the viscosity taken from the hard-sphere form of the mean free path
  (Eq. lambda, second form) and the VHS Chapman-Enskog viscosity, not from the oracle's beta;
- P as the weight t / (tau + t) of the integral solution Eq. (ds) at t = dt - tau, the value the
  paper derives Eq. (p) from, not the simplified 1 - tau/dt;
- the flux of a uniform state as that weight times the Euler flux built here.

A mutant oracle (compiled from a copy of the source with one planted mistake: tau/(2 dt), tau at
the reference temperature, or the flux weight with 2 dt) must fail the same checks."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2305_12071_gb300 import workloads as W


def _tau_vhs(p, rho, T):
    """Relaxation time mu(T)/p in the problem's units from the molecular route: d_ref from the
    hard-sphere mean free path lambda_ref = 1/(sqrt(2) pi d^2 n_ref), the VHS viscosity
    mu_ref = 15 sqrt(pi m k T_ref) / (2 (5 - 2w)(7 - 2w) pi d^2) and mu ~ T^w.  Units: k = m = 1 times
    R (so R = k/m), n = rho / m."""
    R, w, Tref = p["R"], p["omega"], p["T_ref"]
    k, m = R, 1.0
    lam = p["Kn"] * p["L_ref"]
    n_ref = p["rho_ref"] / m
    d2 = 1.0 / (math.sqrt(2.0) * math.pi * lam * n_ref)
    mu_ref = 15.0 * math.sqrt(math.pi * m * k * Tref) / (2.0 * (5 - 2 * w) * (7 - 2 * w) * math.pi * d2)
    mu = mu_ref * (T / Tref) ** w
    return mu / (rho * R * T)


def _p_from_integral_solution(tau, dt):
    """Eq. (p) as the paper derives it: the weight t/(tau + t) of the integral solution Eq. (ds)
    taken at t = dt - tau when dt > tau, no absorption otherwise."""
    if dt <= tau:
        return 0.0
    t = dt - tau
    return t / (tau + t)


def _euler_flux(W5, R=1.0):
    rho, u, v, w, T = W5
    pr = rho * R * T
    E = 0.5 * rho * (u * u + v * v + w * w) + 1.5 * pr
    return np.array([rho * u, rho * u * u + pr, rho * u * v, rho * u * w, u * (E + pr)])


# states and time steps chosen so that P lies well inside (0, 1): 0.1-0.9
_P_CASES = [
    (2e-4, (1.0, 0.0, 0.0, 0.0, 1.0), 2e-3),
    (1e-3, (0.4, 0.3, 0.0, 0.1, 2.5), 2e-2),
    (3e-3, (1.7, -0.2, 0.1, 0.0, 0.6), 1.5e-2),
]


def _check_eq_p(mod):
    for Kn, state, dt in _P_CASES:
        p = W.uniform(n_cells=4, Kn=Kn, ppc_ref=20, state=state, dt=dt, x_max=1.0)
        pr = mod.Oracle(p).prim()
        tau = _tau_vhs(p, state[0], state[4])
        want = _p_from_integral_solution(tau, dt)
        assert 0.05 < want < 0.95, (Kn, want)
        np.testing.assert_allclose(pr["P"], want, rtol=1e-11)
        # dt <= tau on the other side: nothing is absorbed (exactly zero)
        q = mod.Oracle(dict(p, dt=0.9 * tau)).prim()["P"]
        assert np.all(q == 0.0)


def _check_flux_weight(mod):
    for flux in ("gks_eq", "kfvs"):
        for Kn, W5, dt in _P_CASES:
            p = W.base(Kn=Kn, n_cells=100, flux_mode=flux, dt=dt)
            F = mod.wave_flux(p, W5, W5)
            # a uniform state is its own interface equilibrium; its KFVS halves sum to Euler
            tau_f = _tau_vhs(p, W5[0], W5[4])
            Pf = _p_from_integral_solution(tau_f, dt)
            euler = _euler_flux(W5)
            np.testing.assert_allclose(F, Pf * euler, rtol=1e-11, atol=1e-14 * np.abs(euler).max())
            assert np.all(mod.wave_flux(dict(p, dt=0.95 * tau_f), W5, W5) == 0.0)


def test_eq_p_equals_integral_solution_weight(oracle_mod):
    _check_eq_p(oracle_mod)


def test_flux_weight_equals_integral_solution_weight(oracle_mod):
    _check_flux_weight(oracle_mod)


def test_absorbed_fraction_follows_closed_form_p(oracle_mod):
    # the absorption draws use that P: absorbed / arrived ~ Binomial(n, P(closed form))
    Kn, state, dt = _P_CASES[0]
    p = W.uniform(n_cells=10, Kn=Kn, ppc_ref=4000, state=state, dt=dt, x_max=1.0)
    o = oracle_mod.Oracle(p)
    o.step(2)
    n_before = o.num_particles()
    rho = o.prim()["rho"]
    T = o.prim()["T"]
    Pc = np.array([_p_from_integral_solution(_tau_vhs(p, r, t), dt) for r, t in zip(rho, T)])
    o.step(1)
    nabs = o.counters()["nabs"].sum()
    P = float(Pc.mean())
    assert abs(nabs - P * n_before) < 5 * math.sqrt(n_before * P * (1 - P))


# ------------------------------------------------------------------ planted mistakes
_MUTANTS = {
    # P = 1 - tau/(2 dt)
    "half_tau": (r"return 1\.0 - tau / c->dt;", "return 1.0 - tau / (2.0 * c->dt);"),
    # tau taken at the reference temperature instead of the cell's
    "tau_at_Tref": (r"double tau = mu_of_T\(p, c, q->T\) / \(q->rho \* p->R \* q->T\);",
                    "double tau = mu_of_T(p, c, p->T_ref) / (q->rho * p->R * q->T);"),
    # flux weight with 2 dt
    "flux_half": (r"Pf = 1\.0 - tauf / c->dt;", "Pf = 1.0 - tauf / (2.0 * c->dt);"),
}


class _MutantOracle:
    """The oracle module's Oracle / wave_flux calls routed to a mutant build of the C source."""

    def __init__(self, mod, lib):
        self._mod, self._lib = mod, lib

    def _swap(self, fn, *a, **kw):
        saved = self._mod._lib
        self._mod._lib = self._lib
        try:
            return fn(*a, **kw)
        finally:
            self._mod._lib = saved

    def Oracle(self, p):
        mod = self

        class _O:
            def __init__(self):
                self._o = mod._swap(mod._mod.Oracle, p)

            def prim(self):
                return mod._swap(self._o.prim)

            def __del__(self):
                try:
                    mod._swap(self._o.__del__)
                    self._o.h = None
                except Exception:
                    pass
        return _O()

    def wave_flux(self, *a, **kw):
        return self._swap(self._mod.wave_flux, *a, **kw)


def _build_mutant(oracle_mod, tmp_path, name):
    pat, rep = _MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle_mod.__file__), "duwp_oracle.c")).read()
    mutated, n = re.subn(pat, rep, src)
    assert n == 1, f"mutation {name} did not apply"
    cpath = tmp_path / f"mut_{name}.c"
    cpath.write_text(mutated)
    so = tmp_path / f"libmut_{name}.so"
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", str(so), str(cpath), "-lm"], check=True)
    real = oracle_mod.lib()                       # argtypes of the real build, copied onto the mutant
    lib = ctypes.CDLL(str(so))
    for nm in dir(real):
        if nm.startswith("ora_"):
            f, g = getattr(real, nm), getattr(lib, nm)
            if getattr(f, "argtypes", None) is not None:
                g.argtypes = f.argtypes
            g.restype = f.restype
    return lib


@pytest.mark.parametrize("name,check", [("half_tau", _check_eq_p), ("tau_at_Tref", _check_eq_p),
                                        ("flux_half", _check_flux_weight)])
def test_planted_mistakes_fail_the_pins(oracle_mod, tmp_path, name, check):
    lib = _build_mutant(oracle_mod, tmp_path, name)
    with pytest.raises(AssertionError):
        check(_MutantOracle(oracle_mod, lib))
