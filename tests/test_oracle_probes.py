"""Pins of the oracle's pressure sensors and wave-height gauges (the sensors
P_i and gauges H_i of Sec. 4.3), against what the mathematics fixes:

  - the kernel has unit integral and radial symmetry, so the kernel sum w of
    a full lattice is the lattice number density times the particle volume
    (about 1), and on the face of a half-space it is 1/2;
  - a Shepard average reproduces constants exactly, and linear fields at
    points where the weights are symmetric -- the hydrostatic pressure of a
    tank at rest, whose closed form is rho0 g (H - z) (plus the air column's
    weight in the two-phase tank);
  - with one particle the average is that particle's pressure, and its
    weight V W(r) vanishes at r >= 2h;
  - the gauge of a flat lattice block finds the face of the continuum block,
    half a spacing above the top layer (w = 1/2 there by the same symmetry),
    z_lo for a dry line and the top sample for a line that ends under water.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2110_02621_gb300 import scenes as S

G = 9.81


def _free_scene(pos, rho0=1000.0, dp=0.01, dim=3, lo=(-0.2, -0.2, -0.2), hi=(0.2, 0.2, 0.2)):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    return S.Scene(name="free", dp=dp, h=1.3 * dp, c0=10.0, g=(0.0, 0.0, 0.0), lo=lo, hi=hi,
                   phases=[S.Phase(rho0=rho0, eos="linear", z_top=0.0)], fluid_pos=pos,
                   fluid_vel=np.zeros_like(pos), fluid_phase=np.zeros(len(pos), np.int32),
                   wall_pos=np.zeros((0, 3)), dim=dim)


@pytest.fixture(scope="module")
def tank():
    sc = S.still_water_tank((20, 20, 20), dp=0.01)
    return sc, oracle.OracleSim(sc)


def test_kernel_sum_inside_is_the_lattice_number_density(tank):
    """At an interior lattice node, w = sum_j (m/rho_j) W_ij = sigma0 dx^3 to
    within the density's variation over the support (hydrostatic rho_j)."""
    sc, o = tank
    node = np.array([[0.105, 0.105, 0.105]])
    p, w = o.probe_pressure(node)
    # the hydrostatic density at the node (Tait); the linear variation of
    # rho_j over the symmetric support cancels to first order
    rho = oracle.eos_rho(1000.0 * G * (0.2 - 0.105), sc.phases[0], sc.c0)
    expect = oracle.lattice_sigma0(0.01, 0.013) * 0.01 ** 3 * 1000.0 / rho
    assert w[0] == pytest.approx(expect, rel=1e-6)
    assert abs(w[0] - 1.0) < 1e-2


def test_kernel_sum_on_the_free_surface_is_one_half(tank):
    """The face of a half-space of uniform particles is dx/2 above the top
    layer (0.195 m); a symmetric kernel of unit integral gives 1/2 there."""
    _, o = tank
    pts = np.array([[0.105, 0.105, 0.2], [0.1, 0.1, 0.2], [0.0732, 0.1111, 0.2]])
    _, w = o.probe_pressure(pts)
    assert np.all(np.abs(w - 0.5) < 5e-3)  # the lattice's discretisation of the half-space


def test_pressure_sensor_reads_the_hydrostatic_pressure(tank):
    """Interior points (>= 2h from every face): the Shepard average of the
    hydrostatic field rho0 g (H - z), H = 0.2 m.  Lattice nodes and cell
    centres have symmetric weights; arbitrary points are off by a lattice
    moment, well under 1e-3 rho0 g H."""
    _, o = tank
    pts = np.array([[0.105, 0.105, 0.105], [0.1, 0.1, 0.1], [0.1032, 0.0977, 0.0871],
                    [0.05, 0.15, 0.05], [0.1234, 0.0567, 0.1421]])
    p, _ = o.probe_pressure(pts)
    expect = 1000.0 * G * (0.2 - pts[:, 2])
    scale = 1000.0 * G * 0.2
    sym = np.array([True, True, False, True, False])
    assert np.all(np.abs(p - expect)[sym] < 1e-4 * scale)
    assert np.all(np.abs(p - expect) < 1e-3 * scale)


def test_sensor_of_a_uniform_field_is_exact():
    """A constant pressure is reproduced exactly wherever w > 0; w scales
    with rho0/rho (V_j = m/rho_j)."""
    sc = S.still_water_tank((12, 10, 8), dp=0.01)
    rho = np.full(sc.n_fluid, 1003.0)
    o = oracle.OracleSim(sc, rho=rho)
    p_j = o.fluid()["p"]
    assert np.ptp(p_j) == 0.0
    pts = np.array([[0.06, 0.05, 0.04], [0.0, 0.0, 0.0], [0.119, 0.1, 0.08], [0.02, 0.03, 0.09]])
    p, w = o.probe_pressure(pts)
    assert np.all(w > 0)
    assert np.allclose(p, p_j[0], rtol=1e-14, atol=0)
    o1 = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1000.0))
    _, w1 = o1.probe_pressure(pts)
    assert np.allclose(w, w1 * 1000.0 / 1003.0, rtol=1e-14)


def test_sensor_with_one_particle():
    """One particle: p_bar is its pressure, w = V W(r), zero at r >= 2h;
    r = 0 is included."""
    dp, h = 0.01, 0.013
    sc = _free_scene([[0.01, 0.02, 0.03]], dp=dp)
    o = oracle.OracleSim(sc, rho=np.array([1002.0]))
    pj = o.fluid()["p"][0]
    assert pj == pytest.approx(10.0 ** 2 * 2.0)
    r = np.array([0.0, 0.3 * h, 1.1 * h, 1.999 * h, 2.001 * h, 3.0 * h])
    pts = np.array([0.01, 0.02, 0.03]) + np.outer(r, np.array([1.0, 2.0, -2.0]) / 3.0)
    p, w = o.probe_pressure(pts)
    V = 1000.0 * dp ** 3 / 1002.0
    for k, rk in enumerate(r):
        if rk < 2 * h:
            assert w[k] == pytest.approx(V * oracle.W(rk, h), rel=1e-12)
            assert p[k] == pytest.approx(pj, rel=1e-14)
        else:
            assert w[k] == 0.0 and p[k] == 0.0


def test_sensor_with_two_particles_is_their_weighted_mean():
    """Two particles at equal distance: the plain mean of their pressures."""
    sc = _free_scene([[0.0, 0.0, -0.005], [0.0, 0.0, 0.005]])
    o = oracle.OracleSim(sc, rho=np.array([1001.0, 1001.0 + 1e-9]))
    o2 = oracle.OracleSim(sc, rho=np.array([1000.5, 1003.0]))
    pj = o2.fluid()["p"]
    p, _ = o2.probe_pressure(np.array([[0.003, -0.004, 0.0]]))
    V = 1000.0 * 1e-6 / np.array([1000.5, 1003.0])
    assert p[0] == pytest.approx((pj * V).sum() / V.sum(), rel=1e-14)
    o.close()


def test_particles_outside_the_grid_are_not_sampled():
    """The grid of 2h cells from lo = -0.2 m ends at -0.2 + 16 * 0.026 =
    0.216 m; a particle at z = 0.225 m is outside it."""
    sc = _free_scene([[0.0, 0.0, 0.19], [0.0, 0.0, 0.225]], hi=(0.2, 0.2, 0.2))
    o = oracle.OracleSim(sc, rho=np.array([1001.0, 1004.0]))
    assert o.diagnostics()[7] == 1.0
    p, w = o.probe_pressure(np.array([[0.0, 0.0, 0.2], [0.0, 0.0, 0.24]]))
    assert p[0] == pytest.approx(10.0 ** 2 * 1.0, rel=1e-14)  # the in-grid particle alone
    assert w[1] == 0.0 and p[1] == 0.0  # only the escaped particle is within 2h


def test_gauge_finds_the_face_of_a_flat_block():
    """A 24 x 16 x 12 block (dx = 0.01, top layer at 0.115 m): the face of the
    continuum block is at 0.12 m; the line's orientation is checked by the
    unequal extents (a gauge over x = 0.2 is outside the block)."""
    sc = S.still_water_tank((24, 16, 12), dp=0.01, wall_height=0.2)
    o = oracle.OracleSim(sc)
    g = np.array([[0.12, 0.08, 0.0, 0.3], [0.0731, 0.0213, -0.05, 0.25],
                  [0.2, 0.08, 0.0, 0.3],    # inside: the block spans 0.24 m in x
                  [0.12, 0.2, 0.0, 0.3],    # dry: beyond the block in y
                  [0.12, 0.08, 0.0, 0.06],  # ends under water: the top sample
                  [0.5, 0.5, 0.0, 0.3]])    # dry
    H = o.gauge_height(g, 0.0025)
    assert abs(H[0] - 0.12) < 1e-3 * 0.01 * 10
    assert abs(H[1] - 0.12) < 1e-4
    assert abs(H[2] - 0.12) < 1e-4
    assert H[3] == 0.0
    assert H[4] == pytest.approx(0.06, abs=1e-15)
    assert H[5] == 0.0
    # refining the sampling moves the interpolated crossing by far less than dz
    H8 = o.gauge_height(g[:2], 0.0025 / 8)
    assert np.all(np.abs(H8 - H[:2]) < 0.02 * 0.01)


def test_gauge_of_a_falling_column_drops():
    """Causality of the gauge under the oracle's own dynamics: a released
    column only loses height at its centre line during the first steps."""
    sc = S.dam_break(tank=(0.4, 0.1, 0.3), column=(0.1, 0.1, 0.1), dp=0.01, layers=3)
    o = oracle.OracleSim(sc)
    g = np.array([[0.05, 0.05, 0.0, 0.2]])
    H0 = o.gauge_height(g, 0.0025)[0]
    assert abs(H0 - 0.1) < 2e-4
    o.step(200)
    assert o.gauge_height(g, 0.0025)[0] < H0


def test_2d_two_phase_tank_sensors_and_gauge():
    """2-D two-phase tank (Sec. 4.1): water to H = 0.5 m under air to 2H.
    The gauge counts water only, so it finds the water surface; sensors read
    rho_w g (H - z) + rho_a g H in the water and rho_a g (2H - z) in the air."""
    sc = S.two_phase_hydrostatic_tank_2d(dx=0.02)
    o = oracle.OracleSim(sc)
    H = o.gauge_height(np.array([[0.51, 0.0, 0.0, 1.0], [0.25, 0.0, 0.1, 0.9]]), 0.005)
    assert np.all(np.abs(H - 0.5) < 2e-4)
    zw = np.array([0.11, 0.2, 0.33, 0.4])
    za = np.array([0.65, 0.8, 0.9])
    pts = np.array([[0.5, 0.0, z] for z in np.concatenate([zw, za])])
    p, w = o.probe_pressure(pts)
    exp = np.concatenate([1000.0 * G * (0.5 - zw) + 1.0 * G * 0.5, 1.0 * G * (1.0 - za)])
    assert np.all(np.abs(p - exp) < 1e-3 * 1000.0 * G * 0.5)
    assert np.all(np.abs(w - 1.0) < 2e-2)
    # in the air the scale is the air column's weight
    assert np.all(np.abs(p[len(zw):] - exp[len(zw):]) < 0.05 * 1.0 * G * 0.5)
    # on the floor face, half the disc: 1/2 of rho0/rho at the bottom
    _, w_face = o.probe_pressure(np.array([[0.5, 0.0, 0.0]]))
    rho_b = oracle.eos_rho(1000.0 * G * 0.5 + 1.0 * G * 0.5, sc.phases[0], sc.c0)
    assert abs(w_face[0] - 0.5 * 1000.0 / rho_b) < 5e-3
    assert math.isfinite(p.sum())
