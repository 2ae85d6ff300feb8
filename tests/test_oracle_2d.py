"""Pins of the oracle's 2-D form (the paper's 2-D test case of Sec. 4.1):
the 2-D Wendland C2 normalisation and derivative, the 2-D lattice number
density, the paper's printed total energy of the hydrostatic tank, and a
still 2-D tank staying hydrostatic."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2110_02621_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hydrostatic_tank_2d.json")


@pytest.mark.parametrize("h", [0.013, 1.3])
def test_wendland_2d_unit_integral(h):
    """int_0^{2h} W(r) 2 pi r dr = 1 (Simpson, 4000 intervals)."""
    n = 4000
    r = np.linspace(0.0, 2.0 * h, n + 1)
    f = np.array([oracle.W(x, h, 2) * 2.0 * math.pi * x for x in r])
    w = np.ones(n + 1)
    w[1:-1:2], w[2:-1:2] = 4.0, 2.0
    assert (2.0 * h / n) / 3.0 * (w * f).sum() == pytest.approx(1.0, abs=1e-10)


def test_wendland_2d_derivative_and_support():
    h = 0.013
    for q in (0.1, 0.7, 1.3, 1.9):
        r, e = q * h, 1e-7 * h
        fd = (oracle.W(r + e, h, 2) - oracle.W(r - e, h, 2)) / (2 * e)
        assert oracle.dWdr(r, h, 2) == pytest.approx(fd, rel=1e-6)
    assert oracle.W(2 * h, h, 2) == 0.0 and oracle.dWdr(2 * h, h, 2) == 0.0
    # the 2-D and 3-D kernels share their shape: W2/W3 = (7/(4 pi h^2)) / (21/(16 pi h^3))
    assert oracle.W(0.5 * h, h, 2) / oracle.W(0.5 * h, h) == pytest.approx(4.0 * h / 3.0, rel=1e-14)


def test_lattice_number_density_2d_tends_to_the_integral():
    """sigma0 dx^2 -> 1 as h/dx grows (the lattice sum approximates the integral)."""
    dx = 1.0
    errs = [abs(oracle.lattice_sigma0(dx, k * dx, 2) * dx * dx - 1.0) for k in (1.3, 2.6, 5.2)]
    assert errs[0] < 2e-2 and errs[1] < errs[0] and errs[2] < errs[1] and errs[2] < 2e-5


def test_paper_total_energy_of_the_hydrostatic_tank():
    """The water of the Sec. 4.1 tank (L = 1 m, H = 0.5 m) on the (k + 1/2) dx
    lattice holds exactly the paper's T_tot = rho g L H^2 / 2 = 1226.25 J per
    unit depth: sum_k (k + 1/2) dx = H^2 / (2 dx) for H = n dx, so the 2-D
    particle mass m = rho0 dx^2 and the potential energy -sum m g.r give it
    without discretisation error."""
    ref = json.load(open(GOLDEN))
    for dx in (0.01, 0.005):
        sc = S.dam_break_2d(tank=(ref["L_m"], 1.0), column=(ref["L_m"], ref["H_m"]), dx=dx)
        sc.g = (0.0, 0.0, -ref["g"])
        o = oracle.OracleSim(sc)
        d = o.diagnostics()
        assert d[0] == pytest.approx(ref["rho_w"] * ref["L_m"] * ref["H_m"], rel=1e-12)  # mass per depth
        assert d[5] == pytest.approx(ref["T_tot_J"], rel=1e-12)
        o.close()


def test_still_water_2d_stays_hydrostatic():
    """A 2-D water column at rest keeps p = rho0 g (H - z) within 8 % of rho0 g H
    over 200 steps, with no particle crossing the walls.  (On the lattice at
    h = 1.3 dx the discrete pressure force falls about 5 % short of rho0 g --
    a_z = -0.5 m/s^2 in the interior at the start, in 3-D as in 2-D -- so the
    column settles with a pressure that much above the continuum value.)"""
    sc = S.dam_break_2d(tank=(0.2, 0.2), column=(0.2, 0.1), dx=0.01, reinit_every=20)
    H = 0.1
    o = oracle.OracleSim(sc)
    o.step(200)
    f = o.fluid()
    p_ref = 1000.0 * 9.81 * (H - f["x"][:, 2])
    interior = f["x"][:, 2] < H - 3 * sc.dp
    assert np.abs(f["p"][interior] - p_ref[interior]).max() < 0.08 * 1000.0 * 9.81 * H
    assert f["x"][:, 2].min() > 0.0 and f["x"][:, 0].min() > 0.0 and f["x"][:, 0].max() < 0.2
    assert np.abs(f["x"][:, 1]).max() == 0.0  # stays in its plane
