"""Seeded synthetic problem generators (plain dicts) shared by the CUDA path and the oracle.

This module holds no DUWP arithmetic: it only shapes inputs the way the paper's
test cases are shaped (Sec. 4: argon shock structures and Sod tubes; Table of
Sec. 4.2 for the Sod states) and the way the benchmark workloads are specified
(batches of uneven shocks, a large Mach-8 shock, a Poisson serving mix).  The
downstream state of a shock is the Rankine-Hugoniot jump of the upstream one --
that is how a steady shock-structure problem is posed, not part of the method.

A problem dict carries: gas (gamma, Pr, R), VHS (omega, alpha), reference state
and Knudsen number (rho_ref, T_ref, Kn, L_ref; lambda_ref = Kn * L_ref), mesh
(x_min, x_max, n_cells), time step (dt, or cfl when dt <= 0), the two initial
states left/right = (rho, u, v, w, T) split at x_split, boundary kinds
(inout, specular, periodic, vacuum), particles per cell at the reference density
(ppc_ref), particle precision ('fp64' | 'fp32'), options (eps_mode, flux_mode,
ntc_rate), seed and avg_start.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 5.0 / 3.0


def rankine_hugoniot(mach: float, gamma: float = GAMMA):
    """Density, pressure and temperature ratios across a normal shock of upstream Mach number `mach`."""
    m2 = mach * mach
    r = (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p = (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    return r, p, p / r


def base(**kw) -> dict:
    d = dict(gamma=GAMMA, Pr=2.0 / 3.0, R=1.0, omega=0.81, alpha=1.0, rho_ref=1.0, T_ref=1.0,
             Kn=1.0, L_ref=1.0, x_min=0.0, x_max=1.0, n_cells=100, dt=0.0, cfl=0.5,
             left=(1.0, 0.0, 0.0, 0.0, 1.0), right=(1.0, 0.0, 0.0, 0.0, 1.0), x_split=0.5,
             bc_left="inout", bc_right="inout", ppc_ref=100.0, precision="fp64",
             eps_mode="eps1", flux_mode="gks_eq", ntc_rate="particle", seed=1, avg_start=0)
    d.update(kw)
    return d


def shock(mach: float = 3.0, omega: float = 0.81, n_cells: int = 100, ppc_ref: float = 200.0,
          half_width: float = 25.0, Kn: float = 1.0, precision: str = "fp64", seed: int = 1, **kw) -> dict:
    """Steady normal shock in argon: upstream (1, Ma*sqrt(gamma), 0, 0, 1) on [-W, 0), the
    Rankine-Hugoniot downstream state on [0, W]; the domain is measured in upstream mean
    free paths lambda_ref = Kn * L_ref (L_ref = 1/Kn keeps the domain at +-W lambda)."""
    r, _, t = rankine_hugoniot(mach)
    u1 = mach * math.sqrt(GAMMA)
    lam = 1.0
    L_ref = lam / Kn
    d = base(omega=omega, Kn=Kn, L_ref=L_ref, x_min=-half_width * lam, x_max=half_width * lam,
             n_cells=n_cells, left=(1.0, u1, 0.0, 0.0, 1.0), right=(r, u1 / r, 0.0, 0.0, t),
             x_split=0.0, bc_left="inout", bc_right="inout", ppc_ref=ppc_ref, precision=precision,
             seed=seed)
    d.update(kw)
    return d


def large_shock(mach: float = 8.0, omega: float = 0.68, n_cells: int = 100_000, Kn: float = 0.1,
                ppc_ref: float = 415.0, precision: str = "fp32", seed: int = 4, **kw) -> dict:
    """Mach-8 shock on a unit domain with lambda_ref = Kn (L = 1), split at the middle."""
    r, _, t = rankine_hugoniot(mach)
    u1 = mach * math.sqrt(GAMMA)
    d = base(omega=omega, Kn=Kn, L_ref=1.0, x_min=0.0, x_max=1.0, n_cells=n_cells,
             left=(1.0, u1, 0.0, 0.0, 1.0), right=(r, u1 / r, 0.0, 0.0, t), x_split=0.5,
             bc_left="inout", bc_right="inout", ppc_ref=ppc_ref, precision=precision, seed=seed)
    d.update(kw)
    return d


def sod(n_cells: int = 100, Kn: float = 1e-3, ppc_ref: float = 500.0, precision: str = "fp64",
        seed: int = 1, **kw) -> dict:
    """Sod tube of Sec. 4.2: unit length, (rho,u,T) = (1,0,1) | (0.125,0,0.8), specular walls,
    lambda_ref = Kn at the left state."""
    d = base(omega=0.81, Kn=Kn, L_ref=1.0, x_min=0.0, x_max=1.0, n_cells=n_cells,
             left=(1.0, 0.0, 0.0, 0.0, 1.0), right=(0.125, 0.0, 0.0, 0.0, 0.8), x_split=0.5,
             bc_left="specular", bc_right="specular", ppc_ref=ppc_ref, precision=precision, seed=seed)
    d.update(kw)
    return d


def uniform(n_cells: int = 20, Kn: float = 1.0, ppc_ref: float = 100.0, state=(1.0, 0.3, 0.0, 0.0, 1.0),
            bc: str = "periodic", **kw) -> dict:
    """Uniform Maxwellian gas in a periodic (or walled) box."""
    d = base(Kn=Kn, n_cells=n_cells, left=tuple(state), right=tuple(state), bc_left=bc, bc_right=bc,
             ppc_ref=ppc_ref)
    d.update(kw)
    return d


def config1(precision: str = "fp64") -> dict:
    """Mach-3 argon shock, omega 0.81, [-25,25] upstream mean free paths, 100 cells,
    ~200 particles per upstream cell, CFL 0.5 (500 steps in the headline run)."""
    return shock(3.0, omega=0.81, n_cells=100, ppc_ref=200.0, precision=precision, seed=1, avg_start=100)


def config2(Kn: float = 1e-4, precision: str = "fp32", n_cells: int = 1000, seed: int = 1) -> dict:
    """Sod tube, 1000 cells, ~500 particles per cell at the left state."""
    return sod(n_cells=n_cells, Kn=Kn, ppc_ref=500.0, precision=precision, seed=seed)


def config3_batch(n: int = 64, precision: str = "fp32", cells_range=(100, 4000), ppc_range=(100, 1000),
                  mach_range=(1.2, 8.0), rng_seed: int = 2305_12071) -> list:
    """Uneven batch of shock-structure instances (uniform Mach, cell count and particles per cell)."""
    g = np.random.default_rng(rng_seed)
    out = []
    for i in range(n):
        mach = float(g.uniform(*mach_range))
        cells = int(g.integers(cells_range[0], cells_range[1] + 1))
        ppc = float(g.uniform(*ppc_range))
        d = shock(mach, omega=0.81, n_cells=cells, ppc_ref=ppc, precision=precision, seed=1000 + i)
        out.append(d)
    return out


def config4(precision: str = "fp32", Kn: float = 0.1, n_cells: int = 100_000, ppc_ref: float = 415.0) -> dict:
    return large_shock(8.0, omega=0.68, n_cells=n_cells, Kn=Kn, ppc_ref=ppc_ref, precision=precision, seed=4)


def serving_mix(duration_s: float = 600.0, rate_hz: float = 50.0, rng_seed: int = 5,
                cells_range=(100, 10_000), ppc_range=(100, 1000), kn_range=(1e-4, 1.0),
                precision: str = "fp32", shock_steps: int = 500, max_requests: int | None = None) -> list:
    """Poisson arrivals of shock and Sod requests: returns [(t_arrival, params, n_steps), ...]."""
    g = np.random.default_rng(rng_seed)
    t = 0.0
    out = []
    while True:
        t += float(g.exponential(1.0 / rate_hz))
        if t > duration_s or (max_requests is not None and len(out) >= max_requests):
            break
        cells = int(round(math.exp(g.uniform(math.log(cells_range[0]), math.log(cells_range[1])))))
        ppc = float(g.uniform(*ppc_range))
        kn = float(math.exp(g.uniform(math.log(kn_range[0]), math.log(kn_range[1]))))
        seed = int(g.integers(1, 2**31))
        if g.uniform() < 0.5:
            mach = float(g.uniform(1.2, 8.0))
            # shock on the unit domain with lambda_ref = Kn
            r, _, tt = rankine_hugoniot(mach)
            u1 = mach * math.sqrt(GAMMA)
            d = base(omega=0.81, Kn=kn, L_ref=1.0, x_min=0.0, x_max=1.0, n_cells=cells,
                     left=(1.0, u1, 0.0, 0.0, 1.0), right=(r, u1 / r, 0.0, 0.0, tt), x_split=0.5,
                     ppc_ref=ppc, precision=precision, seed=seed)
            steps = shock_steps
        else:
            d = sod(n_cells=cells, Kn=kn, ppc_ref=ppc, precision=precision, seed=seed)
            # Sod to t = 0.15 at CFL 0.5: dt = 0.5 dx / (3 sqrt(2))
            dt = 0.5 * (1.0 / cells) / (3.0 * math.sqrt(2.0))
            steps = int(math.ceil(0.15 / dt))
        out.append((t, d, steps))
    return out
