"""Exact solution of the Riemann problem of the 1D Euler equations for an ideal gas.

Written from the mathematics of the ideal-gas Riemann problem (two nonlinear waves
and a contact; pressure in the star region from the root of
f_L(p) + f_R(p) + u_R - u_L = 0 with shock/rarefaction branch functions), as laid
out in Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4.
Used only as a pin of the oracle's continuum limit.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ak, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * ak / (g - 1.0) * ((p / pk) ** e - 1.0), (1.0 / (rho * ak)) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(L, R, g):
    rl, ul, pl = L
    rr, ur, pr = R
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, al, g)
        fr, dr = _fk(p, rr, pr, ar, g)
        f = fl + fr + ur - ul
        pn = p - f / (dl + dr)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) < 1e-14 * p:
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, al, g)
    fr, _ = _fk(p, rr, pr, ar, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(L, R, g, xi: np.ndarray):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = L
    rr, ur, pr = R
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(L, R, g)
    out = np.zeros((len(xi), 3))
    for k, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    out[k] = (rl, ul, pl)
                else:
                    r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                    out[k] = (r, us, ps)
            else:  # left rarefaction
                shl = ul - al
                asl = al * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - asl
                if s <= shl:
                    out[k] = (rl, ul, pl)
                elif s >= stl:
                    out[k] = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
                    out[k] = (rl * c ** (2 / (g - 1)), 2 / (g + 1) * (al + (g - 1) / 2 * ul + s),
                              pl * c ** (2 * g / (g - 1)))
        else:  # right of contact
            if ps > pr:  # right shock
                sr = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    out[k] = (rr, ur, pr)
                else:
                    r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                    out[k] = (r, us, ps)
            else:  # right rarefaction
                shr = ur + ar
                asr = ar * (ps / pr) ** ((g - 1) / (2 * g))
                st = us + asr
                if s >= shr:
                    out[k] = (rr, ur, pr)
                elif s <= st:
                    out[k] = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
                    out[k] = (rr * c ** (2 / (g - 1)), 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s),
                              pr * c ** (2 * g / (g - 1)))
    return out
