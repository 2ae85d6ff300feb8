"""Pins of the oracle's periodic axes (the periodic fluid-only box in which
the method's pair antisymmetry conserves total momentum to round-off):

  - a lattice filling a periodic box has no boundary: every particle sees the
    full-lattice number density sigma0 (computed by an independent lattice
    sum), and at uniform density it is at rest (zero rates);
  - a jittered, moving periodic box conserves total momentum to round-off
    over many steps, with particles crossing the faces;
  - translating every particle by the same vector (modulo the period) leaves
    every rate unchanged;
  - a particle's neighbours near a face are the brute-force nearest-image set;
  - a period that is not a whole number (>= 3) of 2h cells is refused.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2110_02621_gb300 import scenes as S


def test_full_periodic_lattice_has_the_lattice_number_density_everywhere():
    sc = S.periodic_box()
    o = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1000.0))
    sig = o.fluid()["sigma"]
    s0 = oracle.lattice_sigma0(sc.dp, sc.h)
    assert np.allclose(sig, s0, rtol=1e-12, atol=0)
    drho, a = o.rates()
    assert np.abs(drho).max() < 1e-9 * 1000.0
    assert np.abs(a).max() < 1e-9


@pytest.mark.parametrize("eos", ["linear", "tait"])
def test_periodic_box_conserves_momentum_to_round_off(eos):
    sc = S.periodic_box(jitter=0.3, vel_scale=0.2, rho_jitter=0.003, eos=eos, mu=1e-3)
    o = oracle.OracleSim(sc)
    m = 1000.0 * sc.dp ** 3
    f0 = o.fluid()
    P0 = m * f0["v"].sum(axis=0)
    scale = m * np.abs(f0["v"]).sum()
    o.step(60, 2e-4)
    f = o.fluid()
    P = m * f["v"].sum(axis=0)
    assert np.abs(P - P0).max() < 1e-12 * scale
    # particles crossed the faces and were wrapped back into [lo, hi)
    assert np.all(f["x"] >= 0.0) and np.all(f["x"] < np.array(sc.hi))
    moved = np.abs(f["x"] - f0["x"]) > 0.5 * np.array(sc.hi)
    assert moved.any()
    assert o.diagnostics()[7] == 0.0


def test_rates_are_invariant_under_a_periodic_translation():
    sc = S.periodic_box(jitter=0.3, vel_scale=0.2, rho_jitter=0.003)
    o1 = oracle.OracleSim(sc)
    d1, a1 = o1.rates()
    shift = np.array([0.0371, -0.0519, 0.0823])
    L = np.array(sc.hi)
    x2 = np.mod(sc.fluid_pos + shift, L)
    o2 = oracle.OracleSim(dataclasses.replace(sc, fluid_pos=x2))
    d2, a2 = o2.rates()
    assert np.abs(d2 - d1).max() < 1e-9 * np.abs(d1).max()
    assert np.abs(a2 - a1).max() < 1e-9 * np.abs(a1).max()


def test_neighbours_across_the_faces_are_the_nearest_images():
    sc = S.periodic_box(jitter=0.3)
    o = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1000.0))
    x = o.fluid()["x"]
    L = np.array(sc.hi)
    corner = int(np.argmin(np.linalg.norm(x, axis=1)))  # next to three faces
    for i in (corner, 0, len(x) // 2):
        f, _ = o.neighbors(i)
        d = x - x[i]
        d -= L * np.floor(d / L + 0.5)
        r = np.linalg.norm(d, axis=1)
        brute = np.where((r > 0) & (r < 2 * sc.h))[0]
        assert np.array_equal(np.sort(f), brute)
        assert len(brute) > 40


def test_a_lone_particle_wraps_around_the_period():
    """A single particle in a periodic box (g = 0, nothing to interact with)
    moves in a straight line: after each step its position is (x0 + v t)
    reduced modulo the period into [lo, hi), across the lower and upper
    faces alike."""
    box = S.periodic_box()
    L = np.array(box.hi) - np.array(box.lo)
    x0 = np.array([[0.2 * L[0], 0.7 * L[1], 0.5 * L[2]]])
    v = np.array([-1.3, 0.9, 0.05]) * L[0]  # m/s: more than one period per second
    sc = dataclasses.replace(box, fluid_pos=x0, fluid_vel=v[None, :], fluid_phase=np.zeros(1, np.int32),
                             rho_init=None, g=(0.0, 0.0, 0.0))
    o = oracle.OracleSim(sc, rho=np.array([1000.0]))
    dt, t = 1e-2, 0.0
    for _ in range(8):
        o.step(10, dt)
        t += 10 * dt
        expect = np.array(box.lo) + np.mod(x0[0] + v * t - np.array(box.lo), L)
        assert np.allclose(o.fluid()["x"][0], expect, rtol=0, atol=1e-12)
    assert t * abs(v[0]) > L[0]  # crossed the lower x face at least once


def test_a_particle_just_below_the_upper_face_stays_in_the_grid():
    """A position one ulp below hi along a periodic axis divides to exactly
    the cell count in floating point; the binning wraps that cell to 0, so the
    particle stays inside the grid and sees its neighbour across the face."""
    box = S.periodic_box(m=(3, 1, 1), dp=0.025)  # a box where x / cs rounds up to the cell count
    L = np.array(box.hi) - np.array(box.lo)
    a = [np.nextafter(box.hi[0], -np.inf), 0.5 * L[1], 0.5 * L[2]]
    b = [0.3 * box.dp, 0.5 * L[1], 0.5 * L[2]]
    sc = dataclasses.replace(box, fluid_pos=np.array([a, b]), fluid_vel=np.zeros((2, 3)),
                             fluid_phase=np.zeros(2, np.int32), rho_init=None, g=(0.0, 0.0, 0.0))
    assert np.floor((a[0] - box.lo[0]) / (2 * box.h)) == round(L[0] / (2 * box.h))  # the rounding case
    o = oracle.OracleSim(sc, rho=np.full(2, 1000.0))
    assert o.diagnostics()[7] == 0.0
    f, _ = o.neighbors(0)
    assert list(f) == [1]


def test_a_period_must_be_whole_cells():
    sc = S.periodic_box()
    bad = dataclasses.replace(sc, hi=(sc.hi[0] + 0.3 * sc.dp, sc.hi[1], sc.hi[2]))
    with pytest.raises(RuntimeError):
        oracle.OracleSim(bad)


@pytest.mark.parametrize("dim", [3, 2])
def test_walls_of_a_periodic_channel_see_no_ends(dim):
    """Floor and roof spanning a periodic x (and y): every wall particle's
    normal is exactly vertical -- an edge at the period's ends would tilt the
    normals there -- and the hydrostatic extrapolation holds at every wall
    particle with fluid support, ends included (nearly incompressible linear
    EOS, as in the non-periodic pin)."""
    sc = S.periodic_channel(dim=dim, eos="linear")
    sc = dataclasses.replace(sc, c0=1e4)
    o = oracle.OracleSim(sc)
    w = o.wall()
    n = w["normal"]
    inner = np.isclose(sc.wall_pos[:, 2], -0.5 * sc.dp) | np.isclose(sc.wall_pos[:, 2], sc.phases[0].z_top + 0.5 * sc.dp)
    assert np.abs(n[:, 0]).max() < 1e-12 and np.abs(n[:, 1]).max() < 1e-12
    assert np.all(np.abs(np.abs(n[inner, 2]) - 1.0) < 1e-12)
    H = sc.phases[0].z_top
    has = w["pw"] != 0.0
    zw = sc.wall_pos[:, 2]
    floor = has & (zw < 0)
    expect = 1000.0 * 9.81 * (H - zw[floor])
    assert floor.sum() > 10
    assert np.max(np.abs(w["pw"][floor] - expect)) < 1e-6 * 1000 * 9.81 * H
