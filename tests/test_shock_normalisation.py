"""The shock-structure normalisations of Sec. 4.1 (Eqs. ma3, ma8) on states whose normalised values
are fixed by the definitions: the inflow state, the outflow state and unit stress / heat flux."""
import math

import numpy as np
import pytest

from paper_2305_12071_gb300 import duwp
from paper_2305_12071_gb300 import workloads as W


def test_ma3_and_ma8_fixed_points():
    r2, _, T2 = W.rankine_hugoniot(8.0)
    up, down = (1.0, 1.0), (r2, T2)
    lam, beta, R = 0.37, 0.36533, 1.0
    p1 = up[0] * R * up[1]
    x = np.array([0.0, 0.5 * math.sqrt(math.pi) * lam, beta * math.pi * lam])
    rho = np.array([up[0], down[0], 0.5 * (up[0] + down[0])])
    T = np.array([up[1], down[1], 0.5 * (up[1] + down[1])])
    Pi = np.array([0.0, p1, 2.0 * R * up[1] * up[0]])
    Q = np.array([0.0, p1 * math.sqrt(2 * R * up[1]), up[0] * (2 * R * up[1]) ** 1.5])
    a = duwp.shock_normalised("ma3", x, rho, T, Pi, Q, up, down, lam, beta, R)
    assert a["x"][1] == pytest.approx(1.0) and a["rho"][0] == 1.0 and a["T"][1] == pytest.approx(T2)
    assert a["Pi"][1] == pytest.approx(1.0) and a["Q"][1] == pytest.approx(1.0)
    b = duwp.shock_normalised("ma8", x, rho, T, Pi, Q, up, down, lam, beta, R)
    assert b["x"][2] == pytest.approx(1.0)
    assert b["rho"][0] == 0.0 and b["rho"][1] == pytest.approx(1.0) and b["rho"][2] == pytest.approx(0.5)
    assert b["T"][0] == 0.0 and b["T"][1] == pytest.approx(1.0) and b["T"][2] == pytest.approx(0.5)
    assert b["Pi"][2] == pytest.approx(1.0) and b["Q"][2] == pytest.approx(1.0)
    with pytest.raises(ValueError):
        duwp.shock_normalised("ma5", x, rho, T, Pi, Q, up, down, lam)
