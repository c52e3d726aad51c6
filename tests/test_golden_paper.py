"""Values the paper prints, read from tests/golden/paper_values.txt (no GPU).

These pin the conventions the oracle and the workloads share: the Courant
number of Sec. 3 (whose printed example only matches without sqrt(d)),
the DoF count per scalar variable of Sec. 3.2, the physical constants of
Sec. 2 / Sec. 3.1 and the background atmosphere's hydrostatic balance.
"""

import math
import os

import numpy as np
import pytest

from oracle import physics as ph
from workloads.cases import courant_dt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _load():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (s.strip() for s in line.split("="))
            vals[k] = float(v)
    return vals


def test_courant_worked_example():
    g = _load()
    c = math.sqrt(g["gamma"] * g["R"] * g["courant_T_ref"])
    C_printed = g["courant_printed"]
    # the paper's numbers: r c dt / H, no sqrt(d)
    C_no_sqrt = g["courant_degree"] * c * g["courant_dt"] / g["courant_H"]
    assert abs(C_no_sqrt - C_printed) < g["courant_printed_tol"]
    # the printed formula with sqrt(3) gives a clearly different number
    assert abs(C_no_sqrt / math.sqrt(3.0) - C_printed) > 1.0
    # the workloads' dt formula inverts C both ways
    dt = courant_dt(3, int(g["courant_degree"]), g["courant_H"], c, C_printed, sqrt_d=False)
    assert abs(dt - g["courant_dt"]) < 0.01
    assert abs(g["courant_H"] / g["courant_degree"] - g["effective_resolution_m"]) < 1e-12


def test_dof_convention():
    g = _load()
    for cells, printed in (
        ("scaling_uniform_cells", "scaling_uniform_unknowns_per_scalar_millions"),
        ("scaling_nonconforming_cells", "scaling_nonconforming_unknowns_per_scalar_millions"),
    ):
        per_scalar = g[cells] * (4 + 1) ** 3 / 1e6
        assert abs(per_scalar - g[printed]) < 0.15
    assert abs(100 * (1 - g["wallclock_nonconforming_s"] / g["wallclock_uniform_s"]) - g["saving_percent_printed"]) < 0.5


def test_constants():
    g = _load()
    assert ph.GRAV == g["g"] and ph.R_GAS == g["R"] and ph.GAMMA == g["gamma"]


@pytest.mark.parametrize("atm", [
    dict(kind="stratified", N=0.01, T_ref=293.15, p_ref=1e5),
    dict(kind="isothermal", T0=250.0, p_ref=1e5),
])
def test_background_is_hydrostatic(atm):
    """dp/dz = -rho g for the background (with the factor g restored in the Sec. 3.1 p formula)."""
    z = np.linspace(0.0, 16e3, 33)
    h = 1e-2
    dp = (ph.background(atm, z + h)[1] - ph.background(atm, z - h)[1]) / (2 * h)
    rho = ph.background(atm, z)[0]
    assert np.abs(dp + rho * ph.GRAV).max() < 1e-6


def test_printed_pressure_formula_is_not_hydrostatic():
    """The formula exactly as printed (g/N^2 instead of g^2/N^2) violates the balance."""
    N2, T, pref = 0.01 ** 2, 293.15, 1e5
    G = (ph.GAMMA - 1) / ph.GAMMA
    rho_ref = pref / (ph.R_GAS * T)
    p = lambda z: pref * (1 - (ph.GRAV / N2) * G * rho_ref / pref * (1 - np.exp(-N2 * z / ph.GRAV))) ** (1 / G)
    rho = lambda z: rho_ref * (p(z) / pref) ** (1 / ph.GAMMA) * np.exp(-N2 * z / ph.GRAV)
    z = 1e3
    dp = (p(z + 0.01) - p(z - 0.01)) / 0.02
    assert abs(dp + rho(z) * ph.GRAV) > 1.0
