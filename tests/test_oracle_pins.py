"""Pins of the FP64 oracle against the mathematics and the paper, not itself.

Each test fixes a value that a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand) would change: closed forms,
invariants, brute force on tiny inputs and special cases.  No GPU needed.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2110_02621_gb300 import scenes as S

G = 9.81


# ----------------------------------------------------------------- kernel
@pytest.mark.parametrize("h", [0.013, 0.5, 1.3])
def test_wendland_unit_integral(h):
    """The 3-D Wendland C2 kernel integrates to one over its support."""
    val, err = integrate.quad(lambda r: 4 * math.pi * r * r * oracle.W(r, h),
                              0.0, 2 * h, epsabs=0, epsrel=1e-13, limit=200)
    assert abs(val - 1.0) < 1e-11


@pytest.mark.parametrize("h", [0.013, 1.3])
def test_wendland_derivative_and_support(h):
    """dW/dr matches a central difference of W; W and W' vanish at 2h;
    W' vanishes at r = 0 (the kernel is smooth at the origin)."""
    assert oracle.W(2 * h, h) == 0.0 and oracle.dWdr(2 * h, h) == 0.0
    assert oracle.W(2.2 * h, h) == 0.0
    assert abs(oracle.dWdr(0.0, h)) == 0.0
    for q in [0.05, 0.4, 1.0, 1.5, 1.95]:
        r, e = q * h, 1e-6 * h
        fd = (oracle.W(r + e, h) - oracle.W(r - e, h)) / (2 * e)
        assert abs(oracle.dWdr(r, h) - fd) <= 1e-7 * abs(fd) + 1e-9 / h ** 4
        assert oracle.W(r, h) > 0.0 and oracle.dWdr(r, h) < 0.0


def test_lattice_number_density_converges_to_integral():
    """sigma^0 dx^3 is a lattice Riemann sum of the unit integral: it tends to
    1 as h/dx grows, and at h = 1.3 dx it lies within 1 %."""
    errs = [abs(oracle.lattice_sigma0(1.0, hr) - 1.0) for hr in (1.3, 1.5, 2.0, 2.5)]
    assert errs[0] < 0.01
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 2e-4


# -------------------------------------------------------- equation of state
def test_linear_eos_closed_form():
    ph = S.Phase(rho0=1000.0, eos="linear")
    assert oracle.eos_p(1000.0, ph, 14.0) == 0.0
    assert oracle.eos_p(1001.0, ph, 14.0) == pytest.approx(196.0, rel=1e-14)
    assert oracle.eos_rho(196.0, ph, 14.0) == pytest.approx(1001.0, rel=1e-15)


def test_tait_eos_closed_form():
    """Tait: p(rho0) = 0, p(2 rho0) = rho0 c^2 (2^7 - 1)/7, dp/drho at rho0 = c^2,
    and the inverse undoes the forward map."""
    ph = S.Phase(rho0=1000.0, eos="tait")
    c = 17.155
    assert oracle.eos_p(1000.0, ph, c) == 0.0
    assert oracle.eos_p(2000.0, ph, c) == pytest.approx(1000.0 * c * c * 127 / 7, rel=1e-13)
    e = 1e-4
    slope = (oracle.eos_p(1000.0 + e, ph, c) - oracle.eos_p(1000.0 - e, ph, c)) / (2 * e)
    assert slope == pytest.approx(c * c, rel=1e-8)
    for p in [-500.0, 0.0, 2943.0, 1e5]:
        assert oracle.eos_p(oracle.eos_rho(p, ph, c), ph, c) == pytest.approx(p, abs=1e-9 * max(1, abs(p)))


# ---------------------------------------------------------- Riemann solver
def test_riemann_equal_states():
    Us, ps, Ub, Pb = oracle.riemann(1000.0, 0.3, 2500.0, 1000.0, 0.3, 2500.0, 14.0)
    assert Us == pytest.approx(0.3, rel=1e-15) and ps == pytest.approx(2500.0, rel=1e-15)


def test_riemann_hand_values():
    """Worked by hand from Eq. (RSsolution) with distinct densities, so a swapped
    weight (rho_L p_L instead of rho_L p_R) or a lost limiter shows."""
    rL, UL, pL, rR, UR, pR, c = 1000.0, 1.0, 100.0, 1.0, 0.0, 10.0, 10.0
    Us, ps, Ub, Pb = oracle.riemann(rL, UL, pL, rR, UR, pR, c)
    assert Ub == pytest.approx(1000.0 / 1001.0, rel=1e-15)
    assert Pb == pytest.approx((1000.0 * 10.0 + 1.0 * 100.0) / 1001.0, rel=1e-15)
    assert Us == pytest.approx(1000.0 / 1001.0 + 0.5 * 90.0 / (10.0 * 500.5), rel=1e-14)
    beta = min(3.0 * 1.0, 10.0)
    assert ps == pytest.approx(Pb + 1000.0 * beta * 1.0 / 1001.0, rel=1e-14)
    # clamp: beta = c when the approach speed exceeds c/3
    _, ps2, _, Pb2 = oracle.riemann(1000.0, 20.0, 0.0, 1000.0, 0.0, 0.0, 10.0)
    assert ps2 == pytest.approx(1000.0 * 1000.0 * 10.0 * 20.0 / 2000.0, rel=1e-14)
    # separating states: no dissipation
    _, ps3, _, Pb3 = oracle.riemann(1000.0, -1.0, 5.0, 1000.0, 1.0, 7.0, 10.0)
    assert ps3 == Pb3
    # no limiter = Eq. (RSatWall)
    _, ps4, _, Pb4 = oracle.riemann(rL, UL, pL, rR, UR, pR, c, limiter=False)
    assert ps4 == Pb4


def test_riemann_pressure_symmetric_in_pair():
    """p* of (i, j) equals p* of (j, i) (states seen along e_ji = -e_ij); this
    is what makes the momentum equation antisymmetric (Sec. 2.2)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        rL, rR = rng.uniform(900, 1100, 2)
        UL, UR = rng.normal(0, 1, 2)
        pL, pR = rng.normal(0, 1000, 2)
        a = oracle.riemann(rL, UL, pL, rR, UR, pR, 12.0)[1]
        b = oracle.riemann(rR, -UR, pR, rL, -UL, pL, 12.0)[1]
        assert a == pytest.approx(b, rel=1e-13, abs=1e-9)


# ---------------------------------------------------------- neighbour search
def _brute_neighbors(x, y, h):
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    return [set(np.nonzero((row < (2 * h) ** 2) & (row > 0))[0].tolist()) for row in d2]


@pytest.mark.parametrize("case", ["random", "on_boundaries"])
def test_neighbor_sets_match_brute_force(case):
    rng = np.random.default_rng(11)
    dp, h = 0.01, 0.013
    cs = 2 * h
    box = np.array([0.2, 0.15, 0.1])
    if case == "random":
        x = rng.uniform(0, 1, (1200, 3)) * box
        xw = rng.uniform(0, 1, (500, 3)) * box
    else:  # many points exactly on cell faces, edges and corners
        k = rng.integers(0, 5, (900, 3)).astype(np.float64)
        x = k * cs + np.where(rng.uniform(size=(900, 3)) < 0.5, 0.0,
                              rng.uniform(0, cs, (900, 3)))
        xw = rng.integers(0, 5, (300, 3)).astype(np.float64) * cs
    sc = S.Scene(name="pts", dp=dp, h=h, c0=10.0, g=(0, 0, 0),
                 lo=(0.0, 0.0, 0.0), hi=tuple((box + 2 * cs).tolist()),
                 phases=[S.Phase(eos="linear")], fluid_pos=x,
                 fluid_vel=np.zeros_like(x),
                 fluid_phase=np.zeros(len(x), np.int32), wall_pos=xw,
                 reinit_every=0)
    o = oracle.OracleSim(sc, rho=np.full(len(x), 1000.0))
    bf, bw = _brute_neighbors(x, x, h), _brute_neighbors(x, xw, h)
    for i in range(len(x)):
        f, w = o.neighbors(i)
        assert set(f.tolist()) == bf[i] and len(f) == len(bf[i])
        assert set(w.tolist()) == bw[i] and len(w) == len(bw[i])


def test_cell_list_properties():
    """Every particle lies inside the box of the cell its key names; the order
    is sorted by (key, id); cell ranges partition the sorted order."""
    sc = S.dam_break(tank=(0.3, 0.12, 0.15), column=(0.1, 0.12, 0.08))
    sc.fluid_pos = sc.fluid_pos + np.random.default_rng(5).uniform(-0.3, 0.3, sc.fluid_pos.shape) * sc.dp
    o = oracle.OracleSim(sc)
    c = o.cells()
    nx, ny, nz = c["dims"]
    cs = 2 * sc.h
    for key_name, order_name, start_name, pos in (("key_f", "order_f", "start_f", sc.fluid_pos),
                                                  ("key_w", "order_w", "start_w", sc.wall_pos)):
        key, order, start = c[key_name], c[order_name], c[start_name]
        k = key.astype(np.int64)
        cx, cy, cz = k % nx, (k // nx) % ny, k // (nx * ny)
        corner = np.asarray(sc.lo) + cs * np.stack([cx, cy, cz], 1)
        assert np.all(pos >= corner - 1e-12) and np.all(pos < corner + cs + 1e-12)
        pairs = list(zip(key[order].tolist(), order.tolist()))
        assert pairs == sorted(pairs)
        assert start[0] == 0 and start[-1] == len(pos) and np.all(np.diff(start) >= 0)
        slot_cell = np.repeat(np.arange(len(start) - 1), np.diff(start))
        assert np.array_equal(slot_cell, k[order])


# ------------------------------------------------------------------ walls
def _floor_patch(n=14, layers=3, dp=0.01):
    """A flat wall slab (n x n x layers) with one fluid layer above it."""
    kx, ky, kz = np.meshgrid(np.arange(n), np.arange(n), np.arange(-layers, 0), indexing="ij")
    wall = (np.stack([kx.ravel(), ky.ravel(), kz.ravel()], 1) + 0.5) * dp
    return wall


def test_flat_wall_normals():
    """Eq. (normalVectors) on a flat slab: +z on the top layer, 0 in the
    middle layer (symmetric support), -z on the bottom layer, away from edges."""
    dp = 0.01
    wall = _floor_patch(dp=dp)
    fluid = (np.array([[7.0, 7.0, 5.0]]) + 0.5) * dp
    sc = S.Scene(name="slab", dp=dp, h=1.3 * dp, c0=10.0, g=(0, 0, 0),
                 lo=(-0.05, -0.05, -0.08), hi=(0.19, 0.19, 0.12),
                 phases=[S.Phase(eos="linear")], fluid_pos=fluid,
                 fluid_vel=np.zeros_like(fluid), fluid_phase=np.zeros(1, np.int32),
                 wall_pos=wall, reinit_every=0)
    n = oracle.OracleSim(sc).wall()["normal"]
    k = np.floor(wall / dp).astype(int)
    inner = (k[:, 0] >= 3) & (k[:, 0] < 11) & (k[:, 1] >= 3) & (k[:, 1] < 11)
    top, mid, bot = inner & (k[:, 2] == -1), inner & (k[:, 2] == -2), inner & (k[:, 2] == -3)
    assert np.allclose(n[top], [0, 0, 1], atol=1e-12)
    assert np.all(n[mid] == 0.0)
    assert np.allclose(n[bot], [0, 0, -1], atol=1e-12)


def test_wall_pressure_uniform_field():
    """g = 0 and uniform density: Eq. (wallPressure) returns the fluid pressure
    exactly, for one phase and (W/rho_f weights) for two phases."""
    sc = S.still_water_tank(n_fluid=(6, 6, 6))
    sc.g = (0.0, 0.0, 0.0)
    o = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1003.0))
    p = oracle.eos_p(1003.0, sc.phases[0], sc.c0)
    pw = o.wall()["pw"]
    has = pw != 0.0
    assert has.sum() > 100
    assert np.allclose(pw[has], p, rtol=1e-13)
    sc2 = S.two_phase_still_tank()
    sc2.g = (0.0, 0.0, 0.0)
    rho = np.where(sc2.fluid_phase == 0, 1000.0 + 0.5 / sc2.c0 ** 2, 1.0 + 0.5 / sc2.c0 ** 2)
    pw2 = oracle.OracleSim(sc2, rho=rho).wall()["pw"]
    has2 = pw2 != 0.0
    assert np.allclose(pw2[has2], 0.5, rtol=1e-12)


def test_wall_pressure_hydrostatic_extrapolation():
    """With a nearly incompressible linear EOS (c0 = 1e4) the hydrostatic start
    has p_f = rho0 g (H - z_f) with rho_f = rho0 + O(1/c0^2); the extrapolation
    then gives p_w = rho0 g (H - z_w) at every wall particle with fluid support,
    for any weights.  A dropped rho_f or a flipped (g . r_wf) sign is off by
    rho0 g dx or more."""
    sc = S.still_water_tank(n_fluid=(8, 8, 8), eos="linear")
    sc.c0 = 1e4
    o = oracle.OracleSim(sc)
    pw = o.wall()["pw"]
    H = sc.phases[0].z_top
    zw = sc.wall_pos[:, 2]
    has = pw != 0.0
    assert has.sum() > 300
    expect = 1000.0 * G * (H - zw[has])
    assert np.max(np.abs(pw[has] - expect)) < 1e-6 * 1000 * G * H


def torn_fluid_under_a_roof(eos="tait"):
    """One fluid particle torn to 0.3 rho0 (tension near the Tait limit) 0.01 m
    below a 3 x 3 patch of roof wall particles: the extrapolated p_w of the wall
    above it is p_f + rho_f g.r_wf = p_f - 0.3 rho0 g dz, below EOS(rho0/2)."""
    dp = 0.01
    xw = np.array([[i * dp, j * dp, dp] for i in (-1, 0, 1) for j in (-1, 0, 1)])
    sc = S.Scene(name="torn", dp=dp, h=1.3 * dp, c0=10.0, g=(0.0, 0.0, -G), lo=(-0.1, -0.1, -0.1),
                 hi=(0.1, 0.1, 0.1), phases=[S.Phase(rho0=1000.0, eos=eos, z_top=0.0)],
                 fluid_pos=np.zeros((1, 3)), fluid_vel=np.zeros((1, 3)),
                 fluid_phase=np.zeros(1, np.int32), wall_pos=xw)
    return sc, np.array([300.0])


def test_wall_pressure_of_two_phases_leaves_out_the_heavy_phase():
    """Sec. 2.3: in multi-phase flow the extrapolation weights are divided by
    the fluid density so that the heavy phase's contribution vanishes.  A wall
    particle midway between a water particle (p = 100 Pa) and an air particle
    (p = 0), g = 0: the water's share of p_w is rho_air / (rho_air +
    rho_water), about 1e-3, where plain kernel weights would give 1/2 (as they
    do, exactly, for two water particles)."""
    phases = [S.Phase(eos="linear", rho0=1000.0, reinit="none"),
              S.Phase(eos="linear", rho0=1.0, reinit="none")]
    d = 0.008
    sc = _pair_scene([-2 * d, 0.0, 0.0], [0.0] * 3, [0.0] * 3, phases, 1, walls=[[-d, 0.0, 0.0]])
    rho = np.array([1001.0, 1.0])  # p_water = c0^2 (1001 - 1000) = 100 Pa, p_air = 0
    pw = oracle.OracleSim(sc, rho=rho).wall()["pw"][0]
    assert 0.0 < pw < 2e-3 * 100.0
    assert pw == pytest.approx(100.0 * 1.0 / (1.0 + 1001.0), rel=1e-12)
    one = _pair_scene([-2 * d, 0.0, 0.0], [0.0] * 3, [0.0] * 3, phases[:1], 0, walls=[[-d, 0.0, 0.0]])
    pw1 = oracle.OracleSim(one, rho=np.array([1001.0, 1000.0])).wall()["pw"][0]
    assert pw1 == pytest.approx(50.0, rel=1e-12)


def test_wall_star_pressure_is_the_acoustic_impedance_average():
    """The fluid-wall pair of Eq. (RSatWall) at rest is the linearised
    (acoustic) Riemann problem between the fluid state (rho_i, p_i) and the
    wall state (rho_w, p_w) with one sound speed: p* = (Z_w p_i + Z_i p_w) /
    (Z_i + Z_w), Z = rho c, each side's pressure weighted by the other side's
    impedance.  One particle 0.9 dx above one wall particle with gravity, so
    that p_w = p_i + rho_i g dz differs from p_i, and a soft linear EOS
    (c0 = 1 m/s) so that rho_w differs from rho_i; p* is read back from the
    particle's acceleration a_z = -2 m_w p* / (rho_i rho_w) dW/dr + g_z."""
    dp, h = 0.01, 0.013
    z = 0.9 * dp
    phases = [S.Phase(eos="linear", rho0=1000.0, reinit="none")]
    sc = S.Scene(name="wallpair", dp=dp, h=h, c0=1.0, g=(0.0, 0.0, -9.81), lo=(-0.05, -0.05, -0.05),
                 hi=(0.05, 0.05, 0.05), phases=phases, fluid_pos=np.array([[0.0, 0.0, z]]),
                 fluid_vel=np.zeros((1, 3)), fluid_phase=np.zeros(1, np.int32),
                 wall_pos=np.array([[0.0, 0.0, 0.0]]), reinit_every=0)
    rho_i = 1050.0
    o = oracle.OracleSim(sc, rho=np.array([rho_i]))
    p_i = 1.0 * (rho_i - 1000.0)
    w = o.wall()
    p_w, rho_w = w["pw"][0], w["rhow"][0, 0]
    assert p_w == pytest.approx(p_i + rho_i * 9.81 * z, rel=1e-12)
    assert rho_w == pytest.approx(1000.0 + p_w, rel=1e-12)
    e = 1e-7 * h
    dWdr = (oracle.W(z + e, h) - oracle.W(z - e, h)) / (2 * e)
    m_w = 1000.0 * dp ** 3
    a_z = o.fluid()["a"][0, 2]
    p_star = (a_z + 9.81) * rho_i * rho_w / (-2.0 * m_w * dWdr)
    assert p_star == pytest.approx((rho_w * p_i + rho_i * p_w) / (rho_i + rho_w), rel=1e-7)

@pytest.mark.parametrize("eos", ["tait", "linear"])
def test_wall_density_is_kept_at_half_the_reference(eos):
    """Below EOS(rho0/2) the wall density is rho0/2 (the Tait inverse has no
    value below -rho0 c^2/gamma: a NaN there stops the run); above it, the
    inverse EOS.  Pinned by the closed forms of both equations of state."""
    sc, rho = torn_fluid_under_a_roof(eos)
    o = oracle.OracleSim(sc, rho=rho)
    w = o.wall()
    ph = sc.phases[0]
    p_f = oracle.eos_p(300.0, ph, sc.c0)
    B = 1000.0 * sc.c0 ** 2 / (7.0 if eos == "tait" else 1.0)
    assert p_f == pytest.approx(B * (0.3 ** 7 - 1.0) if eos == "tait" else -700.0 * sc.c0 ** 2, rel=1e-12)
    centre = 4  # the wall right above the particle
    assert w["pw"][centre] == pytest.approx(p_f - 300.0 * G * 0.01, rel=1e-12)
    p_half = B * (0.5 ** 7 - 1.0) if eos == "tait" else -500.0 * sc.c0 ** 2
    for k in range(9):
        if w["pw"][k] < p_half:
            assert w["rhow"][k, 0] == 500.0
        else:
            assert w["rhow"][k, 0] == pytest.approx(oracle.eos_rho(w["pw"][k], ph, sc.c0), rel=1e-13)
    if eos == "tait":
        assert w["pw"][centre] < -B < p_half  # the inverse EOS would be NaN here
    o.step(5, 1e-5)
    f = o.fluid()
    assert np.all(np.isfinite(f["x"])) and np.all(np.isfinite(f["v"])) and np.all(np.isfinite(f["rho"]))


# -------------------------------------------------------------- continuity
def test_continuity_galilean_and_rest():
    """Uniform density and velocity: d rho/dt = 0; with non-uniform density the
    rate is the same at rest and under a uniform translation."""
    sc = S.jittered_blob(n=(8, 8, 8), vel_scale=0.0)
    sc.fluid_vel = np.tile([0.3, -0.2, 0.1], (sc.n_fluid, 1))
    o = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1002.0))
    drho, _ = o.rates()
    assert np.abs(drho).max() < 1e-9
    rho = 1000.0 * (1 + np.random.default_rng(2).uniform(-0.01, 0.01, sc.n_fluid))
    moving = oracle.OracleSim(sc, rho=rho).rates()[0]
    sc.fluid_vel = np.zeros_like(sc.fluid_vel)
    rest = oracle.OracleSim(sc, rho=rho).rates()[0]
    assert np.abs(rest).max() > 1.0
    assert np.allclose(moving, rest, rtol=1e-10, atol=1e-9)


def test_continuity_uniform_compression():
    """v = -alpha (r - c), uniform density: interior d rho/dt approximates
    -rho div v = 3 alpha rho (lattice sum of r.grad W = -3 within 2.5 %)."""
    sc = S.jittered_blob(n=(12, 12, 12), jitter=0.0, vel_scale=0.0)
    alpha = 0.1
    sc.fluid_vel = -alpha * (sc.fluid_pos - sc.fluid_pos.mean(0))
    drho = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1000.0)).rates()[0]
    k = np.floor(sc.fluid_pos / sc.dp).astype(int)
    inner = np.all((k >= 3) & (k < 9), axis=1)
    ratio = drho[inner] / (3 * alpha * 1000.0)
    assert np.all(np.abs(ratio - 1) < 0.025)


def test_continuity_pressure_diffusion_sign():
    """At rest, a particle holding a higher density (pressure) than all its
    neighbours loses density: the Riemann dissipation term is diffusive."""
    sc = S.jittered_blob(n=(7, 7, 7), jitter=0.0, vel_scale=0.0)
    rho = np.full(sc.n_fluid, 1000.0)
    centre = np.argmin(((sc.fluid_pos - sc.fluid_pos.mean(0)) ** 2).sum(1))
    rho[centre] = 1010.0
    drho = oracle.OracleSim(sc, rho=rho).rates()[0]
    assert drho[centre] < 0
    f, _ = oracle.OracleSim(sc, rho=rho).neighbors(centre)
    assert np.all(drho[f] > 0)


def _pair_scene(x_j, v_i, v_j, phases, phase_j, c0=10.0, g=(0.0, 0.0, 0.0), walls=None):
    """Fluid particle 0 at the origin and particle 1 at x_j, no walls unless
    given; reinitialisation off."""
    dp = 0.01
    fluid = np.array([[0.0, 0.0, 0.0], x_j])
    wall = np.zeros((0, 3)) if walls is None else np.asarray(walls, float)
    return S.Scene(name="pair", dp=dp, h=1.3 * dp, c0=c0, g=g, lo=(-0.05, -0.05, -0.05),
                   hi=(0.05, 0.05, 0.05), phases=phases, fluid_pos=fluid,
                   fluid_vel=np.array([v_i, v_j], float), fluid_phase=np.array([0, phase_j], np.int32),
                   wall_pos=wall, reinit_every=0)


def test_continuity_contact_at_an_interface_moves_with_the_mass_weighted_velocity():
    """Two particles of different phases (rho0 1000 and 500, both at their
    reference density, so at equal pressure) approaching head-on.  At equal
    pressures the Riemann solution of Eq. (RSsolution) puts the contact at
    the density-weighted mean normal velocity, so each particle compresses
    with U_L - U* = rho_R (U_L - U_R) / (rho_L + rho_R): the logarithmic
    density rates stand in the ratio m_j : m_i of the particle masses (here
    1 : 2), whatever the densities.  With the densities of the mixture
    swapped the ratio would be m_j rho_i^2 : m_i rho_j^2 (2 : 1)."""
    phases = [S.Phase(eos="linear", rho0=1000.0, reinit="none"),
              S.Phase(eos="linear", rho0=500.0, reinit="none")]
    u = 0.2
    sc = _pair_scene([0.011, 0.0, 0.0], [u, 0.0, 0.0], [-u, 0.0, 0.0], phases, 1)
    rho = np.array([1000.0, 500.0])
    drho, _ = oracle.OracleSim(sc, rho=rho).rates()
    assert drho[0] > 0 and drho[1] > 0  # both compress
    assert (drho[0] / rho[0]) / (drho[1] / rho[1]) == pytest.approx(500.0 / 1000.0, rel=1e-12)
    # one phase (equal masses): equal logarithmic rates at unequal densities
    # would need unequal pressures; at equal densities the rates are equal
    sc1 = _pair_scene([0.011, 0.0, 0.0], [u, 0.0, 0.0], [-u, 0.0, 0.0], phases[:1], 0)
    d1, _ = oracle.OracleSim(sc1, rho=np.array([1000.0, 1000.0])).rates()
    assert d1[0] == pytest.approx(d1[1], rel=1e-14)


# ---------------------------------------------------------------- momentum
def test_momentum_conserved_pairwise():
    """Fluid only, g = 0, jittered positions, random velocities and densities:
    sum_i m_i a_i = 0 to FP64 round-off (antisymmetry, Sec. 2.2), with the
    viscous term on."""
    sc = S.jittered_blob(n=(10, 10, 10), jitter=0.05, vel_scale=0.5, rho_jitter=0.01)
    sc.phases[0].mu = 0.5
    o = oracle.OracleSim(sc)
    a = o.fluid()["a"]
    m = 1000.0 * sc.dp ** 3
    total = (m * a).sum(0)
    scale = (m * np.abs(a)).sum(0)
    assert np.all(np.abs(total) < 1e-13 * scale)
    d0 = o.diagnostics()
    o.step(20)
    d1 = o.diagnostics()
    assert np.allclose(d1[1:4], d0[1:4], rtol=0, atol=1e-13 * d0[0])


def test_momentum_hydrostatic_interior_balance():
    """Hydrostatic start in a tank: pressure gradient and gravity balance in
    the interior to within the lattice gradient error (5 % of g); a flipped
    pressure-force sign gives 2 g."""
    sc = S.still_water_tank(n_fluid=(10, 10, 10))
    o = oracle.OracleSim(sc)
    f = o.fluid()
    k = np.floor(sc.fluid_pos / sc.dp).astype(int)
    inner = np.all((k >= 3) & (k < 7), axis=1)
    assert np.abs(f["a"][inner]).max() < 0.05 * G
    H = sc.phases[0].z_top
    assert np.allclose(f["p"], 1000.0 * G * (H - sc.fluid_pos[:, 2]), rtol=1e-12, atol=1e-9)


def test_viscosity_laplacian():
    """Morris viscosity on the lattice: a linear shear gives no force in the
    interior, v_x = z^2 gives (mu/rho) 2 within 4 %, uniform motion gives 0."""
    sc = S.jittered_blob(n=(12, 12, 12), jitter=0.0, vel_scale=0.0)
    rho = np.full(sc.n_fluid, 1000.0)
    k = np.floor(sc.fluid_pos / sc.dp).astype(int)
    inner = np.all((k >= 3) & (k < 9), axis=1)
    z = sc.fluid_pos[:, 2]
    mu = 1.0

    def visc(vx):
        sc.fluid_vel = np.zeros((sc.n_fluid, 3))
        sc.fluid_vel[:, 0] = vx
        sc.phases[0].mu = 0.0
        a0 = oracle.OracleSim(sc, rho=rho).fluid()["a"]
        sc.phases[0].mu = mu
        a1 = oracle.OracleSim(sc, rho=rho).fluid()["a"]
        return a1 - a0

    assert np.abs(visc(z)[inner]).max() < 1e-12
    q = visc(z ** 2)[inner]
    assert np.all(np.abs(q[:, 0] / (2 * mu / 1000.0) - 1) < 0.04)
    assert np.abs(q[:, 1:]).max() < 1e-12
    assert np.abs(visc(np.full(sc.n_fluid, 0.7))).max() < 1e-12


# ----------------------------------------------------------------- penalty
def _penalty_scene(z_i, gamma_p=1.0):
    """One fluid particle above two stacked wall particles (normals +z on the
    upper, -z on the lower), g = 0, linear EOS."""
    dp = 0.01
    wall = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, -dp]])
    fluid = np.array([[0.0, 0.0, z_i]])
    sc = S.Scene(name="pen", dp=dp, h=1.3 * dp, c0=10.0, g=(0, 0, 0),
                 lo=(-0.05, -0.05, -0.05), hi=(0.05, 0.05, 0.05),
                 phases=[S.Phase(eos="linear", penalty=True)], fluid_pos=fluid,
                 fluid_vel=np.zeros_like(fluid), fluid_phase=np.zeros(1, np.int32),
                 wall_pos=wall, reinit_every=0, gamma_p=gamma_p)
    return sc


def test_penalty_hand_computed_pair():
    """F_p for a particle 0.3 dx above the upper wall particle.  The upper
    particle (n = +z, delta = 0.6) acts; the lower one (n = -z, distance 1.3 dx,
    delta = 2.6) does not.  Expected value built from the printed factors with
    dW/dr taken by central difference of W."""
    dp, h = 0.01, 0.013
    rho = 1000.5
    z_i = 0.3 * dp
    sc = _penalty_scene(z_i)
    on = oracle.OracleSim(sc, rho=np.array([rho])).fluid()["a"][0]
    sc.phases[0].penalty = False
    off = oracle.OracleSim(sc, rho=np.array([rho])).fluid()["a"][0]
    Fp = on - off
    p_i = 100.0 * (rho - 1000.0)          # c0^2 (rho - rho0)
    rho_w = rho                           # p_w = p_i (g = 0, one fluid neighbour)
    m = 1000.0 * dp ** 3
    delta = 2 * z_i / dp
    lam = (1 - delta) ** 2 / dp
    P = 1.0 * lam * abs(p_i * (-1.0))     # e_iw . n_w = -1
    e = 1e-7 * h
    dWdr = (oracle.W(z_i + e, h) - oracle.W(z_i - e, h)) / (2 * e)
    expect = -2 * m / (rho * rho_w) * P * dp ** 3 / z_i ** 2 * dWdr
    assert Fp[0] == 0.0 and Fp[1] == 0.0
    assert Fp[2] > 0
    assert Fp[2] == pytest.approx(expect, rel=1e-7)
    # strength scales linearly; no force once delta >= 1
    sc2 = _penalty_scene(z_i, gamma_p=2.5)
    on2 = oracle.OracleSim(sc2, rho=np.array([rho])).fluid()["a"][0]
    assert (on2 - off)[2] == pytest.approx(2.5 * Fp[2], rel=1e-12)
    sc3 = _penalty_scene(0.55 * dp)
    on3 = oracle.OracleSim(sc3, rho=np.array([rho])).fluid()["a"][0]
    sc3.phases[0].penalty = False
    off3 = oracle.OracleSim(sc3, rho=np.array([rho])).fluid()["a"][0]
    assert np.all(on3 == off3)


def _penalty_pair_expect(z_i, rho, dp=0.01, h=0.013):
    """F_p of Eq. (SPH_penaltyMethodTerm) on a particle at height z_i above a
    wall particle with n_w = +z (delta = 2 z_i / dx signed), equal fluid and
    wall densities, p = c0^2 (rho - rho0) with c0 = 10; dW/dr by central
    difference of W."""
    p_i = 100.0 * (rho - 1000.0)
    m = 1000.0 * dp ** 3
    delta = 2 * z_i / dp
    lam = (1 - delta) ** 2 / dp if delta < 1 else 0.0
    r = abs(z_i)
    P = lam * abs(p_i)                    # |e_iw . n_w| = 1 on the axis
    e = 1e-7 * h
    dWdr = (oracle.W(r + e, h) - oracle.W(r - e, h)) / (2 * e)
    return -2 * m / (rho * rho) * P * dp ** 3 / r ** 2 * dWdr


def test_penalty_barrier_behind_the_plane():
    """A particle 0.2 dx behind the upper wall particle's plane (between the
    two wall layers), with a second particle 1.1 dx in front making the upper
    wall particle fluid-facing: delta = -0.4 (signed), lambda = 1.4^2 / dx,
    and F_p pushes the particle back along n_w = +z.  Under |delta| it would
    be 0.36 / dx.  The particle in front (delta = 2.2) and the lower wall
    particle (normal away from both) add nothing."""
    dp, rho = 0.01, 1000.5
    sc = _penalty_scene(-0.2 * dp)
    sc.fluid_pos = np.array([[0.0, 0.0, -0.2 * dp], [0.0, 0.0, 1.1 * dp]])
    sc.fluid_vel = np.zeros((2, 3))
    sc.fluid_phase = np.zeros(2, np.int32)
    r2 = np.full(2, rho)
    on = oracle.OracleSim(sc, rho=r2).fluid()["a"]
    sc.phases[0].penalty = False
    off = oracle.OracleSim(sc, rho=r2).fluid()["a"]
    Fp = on - off
    assert Fp[0, 0] == 0.0 and Fp[0, 1] == 0.0
    assert Fp[0, 2] > 0
    assert Fp[0, 2] == pytest.approx(_penalty_pair_expect(-0.2 * dp, rho), rel=1e-7)
    assert np.all(Fp[1] == 0.0)


def test_penalty_only_through_fluid_facing_wall_particles():
    """The same penetrated particle alone: no fluid lies on the side of the
    upper wall particle's normal, so that particle is not fluid-facing and
    the penalty is silent (as it is for the outer wall layers, whose normals
    point away from the fluid)."""
    dp, rho = 0.01, 1000.5
    sc = _penalty_scene(-0.2 * dp)
    on = oracle.OracleSim(sc, rho=np.array([rho])).fluid()["a"][0]
    sc.phases[0].penalty = False
    off = oracle.OracleSim(sc, rho=np.array([rho])).fluid()["a"][0]
    assert np.all(on == off)


def test_penalty_silent_at_rest():
    """In a lattice tank at rest every fluid particle is at least dx from the
    tangent plane of each wall neighbour: switching the penalty on changes
    nothing."""
    sc = S.dam_break(tank=(0.3, 0.12, 0.15), column=(0.1, 0.12, 0.08), penalty=False)
    a0 = oracle.OracleSim(sc).fluid()["a"]
    sc.phases[0].penalty = True
    a1 = oracle.OracleSim(sc).fluid()["a"]
    assert np.array_equal(a0, a1)


# ---------------------------------------------------- density reinitialisation
def test_reinit_lattice_interior_closed_forms():
    """Full lattice support gives sigma = sigma^0, so Eq. (eqrhosum) returns
    rho0 + (rho* - rho0) rho0/rho* and Eq. (eqrhosumnosurface) returns rho0;
    at the blob surface (sigma < sigma^0) the free-surface form keeps
    rho_num <= rho <= rho*."""
    rho_star = 1005.0
    for mode, expect in (("free_surface", 1000.0 + 5.0 * 1000.0 / 1005.0),
                         ("internal", 1000.0)):
        sc = S.jittered_blob(n=(9, 9, 9), jitter=0.0, vel_scale=0.0)
        sc.phases[0].reinit = mode
        o = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, rho_star))
        o.reinit_density()
        f = o.fluid()
        k = np.floor(sc.fluid_pos / sc.dp).astype(int)
        inner = np.all((k >= 2) & (k < 7), axis=1)
        assert np.allclose(f["sigma"][inner], o.sigma0, rtol=1e-13)
        assert np.allclose(f["rho"][inner], expect, rtol=1e-13)
        if mode == "free_surface":
            rho_num = 1000.0 * f["sigma"] / o.sigma0
            assert np.all(f["rho"] >= rho_num - 1e-9) and np.all(f["rho"] <= rho_star + 1e-9)
            assert np.any(f["sigma"] < 0.7 * o.sigma0)


def test_summation_density_lattice():
    """Eq. (densitySummation) on a full lattice: rho = m sigma^0."""
    sc = S.jittered_blob(n=(9, 9, 9), jitter=0.0, vel_scale=0.0, eos="linear")
    sc.phases[0].density = "summation"
    o = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1000.0))
    o.step(1, dt=1e-6)
    f = o.fluid()
    k = np.floor(sc.fluid_pos / sc.dp).astype(int)
    inner = np.all((k >= 2) & (k < 7), axis=1)
    assert np.allclose(f["rho"][inner], 1000.0 * sc.dp ** 3 * o.sigma0, rtol=1e-12)


def test_summation_density_is_completed_by_the_walls():
    """The wall dummy particles continue the fluid lattice (three layers, the
    first dx/2 behind each face), so they complete the kernel support of the
    fluid next to them: in a still-water tank with summation density every
    particle more than 2h below the free surface, those touching the floor, the
    side walls and the corners included, has the interior lattice value
    rho = m sigma^0 of Eq. (densitySummation)."""
    sc = S.still_water_tank(n_fluid=(8, 8, 8), eos="linear")
    sc.phases[0].density = "summation"
    sc.phases[0].reinit = "none"
    o = oracle.OracleSim(sc, rho=np.full(sc.n_fluid, 1000.0))
    o.step(1, dt=1e-7)
    f = o.fluid()
    H = sc.phases[0].z_top
    deep = sc.fluid_pos[:, 2] < H - 2 * sc.h
    at_wall = deep & ((sc.fluid_pos[:, 2] < sc.dp) | (sc.fluid_pos[:, 0] < sc.dp))
    assert at_wall.sum() > 20
    assert np.allclose(f["rho"][deep], 1000.0 * sc.dp ** 3 * o.sigma0, rtol=1e-9)


# -------------------------------------------------------------- integrator
def test_kick_drift_kick_free_fall():
    """A lone particle under gravity: KDK is exact for constant acceleration,
    z = z0 + v0 t + g t^2/2 and v = v0 + g t."""
    x0 = np.array([[0.1, 0.1, 0.5]])
    v0 = np.array([[0.2, 0.0, 1.0]])
    sc = S.Scene(name="fall", dp=0.01, h=0.013, c0=10.0, g=(0.0, 0.0, -G),
                 lo=(-1, -1, -1), hi=(1, 1, 1), phases=[S.Phase(eos="linear")],
                 fluid_pos=x0, fluid_vel=v0, fluid_phase=np.zeros(1, np.int32),
                 wall_pos=np.zeros((0, 3)), reinit_every=0)
    o = oracle.OracleSim(sc, rho=np.array([1000.0]))
    dt, n = 1e-3, 100
    o.step(n, dt=dt)
    f = o.fluid()
    t = n * dt
    assert f["x"][0] == pytest.approx([0.1 + 0.2 * t, 0.1, 0.5 + t - 0.5 * G * t * t], abs=1e-13)
    assert f["v"][0] == pytest.approx([0.2, 0.0, 1.0 - G * t], abs=1e-13)


def test_time_step_limits():
    """dt = min(0.25 h/(c + U_max), 0.25 sqrt(h/|g|)) (Sec. 2.6)."""
    sc = S.still_water_tank(n_fluid=(4, 4, 4))
    o = oracle.OracleSim(sc)
    dt = o.step(1)
    assert dt == pytest.approx(min(0.25 * sc.h / sc.c0, 0.25 * math.sqrt(sc.h / G)), rel=1e-14)
    sc.c0 = 0.2   # below sqrt(g h): the body-force limit wins
    dt2 = oracle.OracleSim(sc).step(1)
    assert dt2 == pytest.approx(0.25 * math.sqrt(sc.h / G), rel=1e-14)
    # the flow speed enters the acoustic limit: a blob translating at
    # |v| = 3 m/s without gravity
    blob = S.jittered_blob(n=(4, 4, 4), vel_scale=0.0)
    blob.g = (0.0, 0.0, 0.0)
    v = np.array([1.0, -2.0, 2.0])
    blob.fluid_vel = np.tile(v, (blob.n_fluid, 1))
    dt3 = oracle.OracleSim(blob, rho=np.full(blob.n_fluid, 1000.0)).step(1)
    assert dt3 == pytest.approx(0.25 * blob.h / (blob.c0 + 3.0), rel=1e-14)


def test_diagnostics_of_a_translating_blob():
    """Sec. 4.1's energies on a blob of N particles of mass m = rho0 dx^3
    translating at v: mass N m, momentum N m v, kinetic energy N m |v|^2 / 2,
    potential energy -N m g . x_mean, U_max = |v|, nothing escaped."""
    blob = S.jittered_blob(n=(5, 4, 3), vel_scale=0.0)
    v = np.array([0.3, -0.4, 1.2])
    blob.fluid_vel = np.tile(v, (blob.n_fluid, 1))
    o = oracle.OracleSim(blob, rho=np.full(blob.n_fluid, 1000.0))
    d = o.diagnostics()
    N, m = blob.n_fluid, 1000.0 * blob.dp ** 3
    g = np.array(blob.g, float)
    assert d[0] == pytest.approx(N * m, rel=1e-13)
    assert np.allclose(d[1:4], N * m * v, rtol=1e-13, atol=0)
    assert d[4] == pytest.approx(0.5 * N * m * (v @ v), rel=1e-13)
    assert d[5] == pytest.approx(-N * m * (g @ blob.fluid_pos.mean(0)), rel=1e-12)
    assert d[6] == pytest.approx(np.sqrt(v @ v), rel=1e-14) and d[7] == 0.0


# ---------------------------------------------------------- whole-step checks
def test_still_water_tank_stays_hydrostatic():
    """Still water (the paper's hydrostatic case, Sec. 4.1, in 3-D): after 200
    steps the interior fluid and the submerged wall pressures stay within 2 %
    of rho0 g depth, no particle crosses a wall, mass is exact, and the initial
    potential energy is rho0 g A H^2 / 2."""
    sc = S.still_water_tank(n_fluid=(10, 10, 10), wall_height=0.15)
    o = oracle.OracleSim(sc)
    d0 = o.diagnostics()
    A, H = 0.1 * 0.1, sc.phases[0].z_top
    assert d0[5] == pytest.approx(1000.0 * G * A * H * H / 2, rel=1e-12)
    assert d0[0] == pytest.approx(1000.0 * A * H, rel=1e-12)
    o.step(200)
    f, w = o.fluid(), o.wall()
    x = f["x"]
    assert np.all(x[:, 0] > 0) and np.all(x[:, 0] < 0.1)
    assert np.all(x[:, 1] > 0) and np.all(x[:, 1] < 0.1) and np.all(x[:, 2] > 0)
    deep = x[:, 2] < H - 3 * sc.dp
    ref = 1000.0 * G * (H - x[deep, 2])
    assert np.max(np.abs(f["p"][deep] - ref)) < 0.02 * 1000.0 * G * H
    zw = sc.wall_pos[:, 2]
    sub = (w["pw"] != 0) & (zw < H - 3 * sc.dp)
    assert np.max(np.abs(w["pw"][sub] - 1000.0 * G * (H - zw[sub]))) < 0.02 * 1000.0 * G * H
    assert o.diagnostics()[0] == d0[0]


# ------------------------------------------------------ tank excitation
def test_excitation_free_particle_closed_form():
    """A lone particle in a tank moving as x = amp sin(w t) (simulated in the
    tank frame, body force g + amp w^2 sin(w t)): x(t) = x0 + v0 t + g t^2/2 +
    amp (w t - sin w t), v(t) = v0 + g t + amp w (1 - cos w t); KDK is second
    order, so 3000 steps of 1e-4 s stay within 1e-8 m (the particle stays
    inside the grid, 40 cells of 2h around its start)."""
    sc = S.jittered_blob(n=(1, 1, 1), jitter=0.0, vel_scale=0.0, margin_cells=40)
    sc.g = (0.0, 0.0, -9.81)
    sc.fluid_vel = np.array([[0.05, 0.0, 0.1]])
    amp, f = np.array([0.1, 0.0, 0.02]), 0.496
    o = oracle.OracleSim(sc, rho=np.array([1000.0]))
    o.set_excitation(amp, f)
    n, dt = 3000, 1e-4
    o.step(n, dt)
    t = o.time
    assert t == pytest.approx(n * dt, rel=1e-12)
    w = 2 * np.pi * f
    g = np.array(sc.g)
    x = sc.fluid_pos[0] + sc.fluid_vel[0] * t + 0.5 * g * t * t + amp * (w * t - np.sin(w * t))
    v = sc.fluid_vel[0] + g * t + amp * w * (1 - np.cos(w * t))
    st = o.fluid()
    assert np.abs(st["x"][0] - x).max() < 1e-8
    assert np.abs(st["v"][0] - v).max() < 1e-7


def test_wall_pressure_extrapolation_with_a_tilted_body_force():
    """With g = (3, 0, -9.81) (a tank accelerating along -x, seen in its frame)
    and the matching linear field p_f = rho0 g.(r_f - r_ref), the extrapolation
    (g.r_wf weighted by rho_f) reproduces p(r_w) = rho0 g.(r_w - r_ref) at every
    supported wall particle, whatever the weights."""
    sc = S.still_water_tank(n_fluid=(8, 8, 8), eos="linear")
    sc.c0 = 1e4
    g = np.array([3.0, 0.0, -9.81])
    sc.g = tuple(g)
    r_ref = np.array([0.0, 0.0, sc.phases[0].z_top])
    p_f = 1000.0 * (sc.fluid_pos - r_ref) @ g
    rho = 1000.0 + p_f / sc.c0 ** 2
    o = oracle.OracleSim(sc, rho=rho)
    pw = o.wall()["pw"]
    has = pw != 0.0
    assert has.sum() > 300
    expect = 1000.0 * (sc.wall_pos[has] - r_ref) @ g
    assert np.max(np.abs(pw[has] - expect)) < 1e-6 * 1000 * 9.81 * 0.1
