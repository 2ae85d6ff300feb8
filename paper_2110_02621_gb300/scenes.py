"""Seeded synthetic particle inputs shaped like the paper's 3-D test cases.

This module only places particles and fills in configuration numbers.  It holds
none of the method's arithmetic (no kernel, no equation of state, no Riemann
solver, no hydrostatic density): both the CUDA library and the CPU oracle take
its output as plain inputs and compute everything else themselves.

Geometry conventions (shared by every generator):
  * particles sit on a cubic lattice at (k + 1/2) * dp;
  * a tank of inner size Lx x Ly x Lz has its inner floor at z = 0 and its
    inner side faces at x = 0, x = Lx, y = 0, y = Ly; it has no roof;
  * wall dummy particles fill ``layers`` lattice layers outside the floor and
    the four side faces, up to the tank height (corners included);
  * the neighbour-grid domain [lo, hi] is the wall bounding box padded by one
    grid cell (2h) on every side, plus head room above the tank, and its
    lower corner lies a further dp/10 below: with cells of 2h = 2.6 dp the
    faces would otherwise pass exactly through lattice sites (every 13th),
    where the cell of a particle that has barely moved is decided by the last
    bit of its coordinate; shifted, every site stays at least dp/10 from a
    face.

Sizes follow the paper's cases (Sec. 4): the smoothing length is h = 1.3 dx
with support radius 2h, g = 9.81 m/s^2, and the sound speed is chosen as
c0 = 10 sqrt(g H) with H the initial depth of the heavy phase.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

G = 9.81
SEED_JITTER = 20211006
SEED_PROBES = 1


@dataclasses.dataclass
class Phase:
    rho0: float = 1000.0
    eos: str = "tait"              # "tait" | "linear"
    density: str = "continuity"    # "continuity" | "summation"
    reinit: str = "free_surface"   # "free_surface" | "internal" | "none"
    penalty: bool = False
    mu: float = 0.0                # dynamic viscosity [Pa s]
    z_top: float = 0.0             # top of this phase's column (hydrostatic init)


@dataclasses.dataclass
class Scene:
    name: str
    dp: float
    h: float
    c0: float
    g: Tuple[float, float, float]
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    phases: List[Phase]
    fluid_pos: np.ndarray            # (N, 3) float64
    fluid_vel: np.ndarray            # (N, 3) float64
    fluid_phase: np.ndarray          # (N,) int32
    wall_pos: np.ndarray             # (M, 3) float64
    gamma_tait: float = 7.0
    gamma_p: float = 1.0
    cfl: float = 0.25
    reinit_every: int = 1
    periodic: Tuple[int, int, int] = (0, 0, 0)
    steps: int = 1
    probes: Optional[np.ndarray] = None   # indices into wall_pos
    rho_init: Optional[np.ndarray] = None  # None: hydrostatic initial density
    sensors: Optional[np.ndarray] = None   # (n, 3) pressure-sensor points
    gauges: Optional[np.ndarray] = None    # (n, 4) wave-gauge lines x, y, z_lo, z_hi
    dim: int = 3                           # 2: particles in the x-z plane y = 0

    @property
    def n_fluid(self) -> int:
        return int(self.fluid_pos.shape[0])

    @property
    def n_wall(self) -> int:
        return int(self.wall_pos.shape[0])


def _count(length: float, dp: float) -> int:
    """Number of lattice sites of spacing dp that fit a length (half rounds up)."""
    return int(math.floor(length / dp + 0.5))


def lattice(n: Tuple[int, int, int], dp: float,
            origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)) -> np.ndarray:
    """Points origin + (k + 1/2) dp for k in [0, n) per axis, x fastest."""
    nx, ny, nz = n
    kx = (np.arange(nx, dtype=np.float64) + 0.5) * dp + origin[0]
    ky = (np.arange(ny, dtype=np.float64) + 0.5) * dp + origin[1]
    kz = (np.arange(nz, dtype=np.float64) + 0.5) * dp + origin[2]
    z, y, x = np.meshgrid(kz, ky, kx, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def tank_walls(inner: Tuple[int, int], height: int, dp: float,
               layers: int = 3) -> np.ndarray:
    """Wall dummy particles of an open-top box tank.

    ``inner`` = (nx, ny) lattice sites across the floor, ``height`` = number
    of lattice layers the side walls rise above the floor.  Returns the
    lattice sites of the padded box [-layers, n + layers) x ... x
    [-layers, height) that are not inside the tank.
    """
    nx, ny = inner
    kx = np.arange(-layers, nx + layers)
    ky = np.arange(-layers, ny + layers)
    kz = np.arange(-layers, height)
    z, y, x = np.meshgrid(kz, ky, kx, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    inside = (x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0)
    keep = ~inside
    k = np.stack([x[keep], y[keep], z[keep]], axis=1).astype(np.float64)
    return (k + 0.5) * dp


def _domain(wall: np.ndarray, fluid: np.ndarray, cell: float,
            head_room: float, dp: float) -> Tuple[tuple, tuple]:
    pts = wall if wall.shape[0] else fluid
    lo = pts.min(axis=0) - cell - 0.1 * dp
    hi = pts.max(axis=0) + cell
    hi[2] += head_room
    return tuple(float(v) for v in lo), tuple(float(v) for v in hi)


def still_water_tank(n_fluid: Tuple[int, int, int] = (20, 20, 20),
                     dp: float = 0.01, wall_height: float = 0.3,
                     layers: int = 3, eos: str = "tait",
                     steps: int = 100) -> Scene:
    """Water block filling the floor of an open box tank, at rest.

    Default: a 20^3 block (8,000 particles, dp = 0.01 m) in a 0.2 x 0.2 m
    tank whose walls rise to 0.3 m, three wall layers.
    """
    nx, ny, nz = n_fluid
    h = 1.3 * dp
    H = nz * dp
    fluid = lattice(n_fluid, dp)
    wall = tank_walls((nx, ny), _count(wall_height, dp), dp, layers)
    lo, hi = _domain(wall, fluid, 2 * h, 2 * h, dp)
    c0 = 10.0 * math.sqrt(G * H)
    return Scene(
        name=f"still_water_tank_{nx}x{ny}x{nz}_dp{dp:g}", dp=dp, h=h, c0=c0,
        g=(0.0, 0.0, -G), lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos=eos, z_top=H)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid),
        fluid_phase=np.zeros(fluid.shape[0], np.int32), wall_pos=wall,
        reinit_every=1, steps=steps)


def dam_break(tank: Tuple[float, float, float] = (1.6, 0.67, 0.6),
              column: Tuple[float, float, float] = (0.4, 0.67, 0.3),
              dp: float = 0.01, layers: int = 3, penalty: bool = True,
              reinit_every: int = 20, steps: int = 2000,
              mu: float = 0.0, n_probes: int = 0, probe_wall: str = "far") -> Scene:
    """Single-phase 3-D dam break: a water column at the x = 0 end of a box.

    Defaults: tank 1.6 x 0.67 x 0.6 m, column 0.4 x 0.67 x 0.3 m, dp = 0.01
    (80,400 fluid and 120,234 wall particles), penalty on, density
    reinitialisation every 20 steps.  With ``n_probes`` > 0 a square grid of
    probe wall particles is chosen on the inner layer of the far wall
    (``probe_wall="far"``, x = Lx side) or of the wall behind the water column
    (``"near"``, x = 0 side) over z in [0, column height].
    """
    ntx, nty, ntz = (_count(v, dp) for v in tank)
    ncx, ncy, ncz = (_count(v, dp) for v in column)
    h = 1.3 * dp
    H = ncz * dp
    fluid = lattice((ncx, ncy, ncz), dp)
    wall = tank_walls((ntx, nty), ntz, dp, layers)
    lo, hi = _domain(wall, fluid, 2 * h, 0.25 * tank[2], dp)
    probes = None
    if n_probes > 0:
        side = int(round(math.sqrt(n_probes)))
        x_in = ntx * dp + 0.5 * dp if probe_wall == "far" else -0.5 * dp
        cand = np.where(np.abs(wall[:, 0] - x_in) < 0.25 * dp)[0]
        cand = cand[(wall[cand, 2] > 0.0) & (wall[cand, 2] < H)
                    & (wall[cand, 1] > 0.0) & (wall[cand, 1] < nty * dp)]
        ky = np.floor(wall[cand, 1] / dp).astype(np.int64)
        kz = np.floor(wall[cand, 2] / dp).astype(np.int64)
        ys, zs = np.unique(ky), np.unique(kz)
        ysel = ys[np.linspace(0, len(ys) - 1, side).round().astype(int)]
        zsel = zs[np.linspace(0, len(zs) - 1, side).round().astype(int)]
        pick = np.isin(ky, ysel) & np.isin(kz, zsel)
        probes = np.sort(cand[pick]).astype(np.int64)
    return Scene(
        name=(f"dam_break_{tank[0]:g}x{tank[1]:g}x{tank[2]:g}"
              f"_col{column[0]:g}x{column[1]:g}x{column[2]:g}_dp{dp:g}"),
        dp=dp, h=h, c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G),
        lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="tait", penalty=penalty, mu=mu,
                      z_top=H)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid),
        fluid_phase=np.zeros(fluid.shape[0], np.int32), wall_pos=wall,
        reinit_every=reinit_every, steps=steps, probes=probes)


def dam_break_obstacle(tank: Tuple[float, float, float] = (3.0, 1.0, 1.6),
                       column: Tuple[float, float, float] = (1.0, 1.0, 0.5),
                       obstacle_lo: Tuple[float, float] = (2.2, 0.3),
                       obstacle_size: Tuple[float, float, float] = (0.16, 0.4, 0.16),
                       dp: float = 0.016, layers: int = 3, penalty: bool = True,
                       reinit_every: int = 1, steps: int = 2000,
                       roof: bool = False) -> Scene:
    """3-D dam break onto a box obstacle standing on the bed, with pressure
    sensors on the obstacle and wave-height gauges along the tank (the
    configuration of Sec. 4.3; the dimensions here are synthetic).

    A water column (``column``, against the x = 0 wall) in an open box tank
    whose walls (1.6 m) stand higher than the surge runs up the far wall (a
    ``roof`` can close it); the obstacle is a solid block of wall particles
    on the lattice of the tank, from (``obstacle_lo``, z = 0) spanning
    ``obstacle_size``.  Density reinitialisation every step, as in the
    paper (Sec. 2.5).  Sensors:
    four points on the obstacle's upstream face (x = face, y = centre, at
    1/8, 3/8, 5/8 and 7/8 of its height) and one at the centre of its top.
    Gauges: vertical lines over the full tank height at x = column/2, column,
    midway to the obstacle and 0.2 m before it, on the tank's centre line.
    Defaults at dp = 0.016 m: 123,039 fluid and 179,962 wall particles.
    """
    ntx, nty, ntz = (_count(v, dp) for v in tank)
    ncx, ncy, ncz = (_count(v, dp) for v in column)
    h = 1.3 * dp
    H = ncz * dp
    fluid = lattice((ncx, ncy, ncz), dp)
    walls = tank_walls((ntx, nty), ntz, dp, layers)
    ox0, oy0 = _count(obstacle_lo[0], dp), _count(obstacle_lo[1], dp)
    onx, ony, onz = (_count(v, dp) for v in obstacle_size)
    if not (ncx < ox0 and ox0 + onx <= ntx and oy0 + ony <= nty and onz < ntz):
        raise ValueError("the obstacle must stand inside the tank, downstream of the column")
    block = lattice((onx, ony, onz), dp, origin=(ox0 * dp, oy0 * dp, 0.0))
    parts = [walls, block]
    if roof:
        parts.append(lattice((ntx + 2 * layers, nty + 2 * layers, layers), dp,
                             origin=(-layers * dp, -layers * dp, ntz * dp)))
    wall = np.concatenate(parts)
    lo, hi = _domain(wall, fluid, 2 * h, 0.0 if roof else 0.2, dp)
    face_x, yc = ox0 * dp, (oy0 + 0.5 * ony) * dp
    top = onz * dp
    sensors = np.array([[face_x, yc, f * top] for f in (0.125, 0.375, 0.625, 0.875)]
                       + [[(ox0 + 0.5 * onx) * dp, yc, top]])
    Lc, xo = ncx * dp, ox0 * dp
    gx = (0.5 * Lc, Lc, 0.5 * (Lc + xo), xo - 0.2)
    gauges = np.array([[x, 0.5 * nty * dp, 0.0, ntz * dp] for x in gx])
    return Scene(
        name=(f"dam_break_obstacle_{tank[0]:g}x{tank[1]:g}x{tank[2]:g}"
              f"_col{column[0]:g}x{column[1]:g}x{column[2]:g}_dp{dp:g}"),
        dp=dp, h=h, c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G),
        lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="tait", penalty=penalty, z_top=H)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid),
        fluid_phase=np.zeros(fluid.shape[0], np.int32), wall_pos=wall,
        reinit_every=reinit_every, steps=steps, sensors=sensors, gauges=gauges)


def two_phase_ramp_cylinder(tank: Tuple[float, float, float] = (1.0, 0.5, 0.5),
                            column: Tuple[float, float, float] = (0.3, 0.5, 0.2),
                            dp: float = 0.005, layers: int = 3,
                            ramp_x0: float = 0.5, ramp_deg: float = 30.0,
                            cyl_xy: Tuple[float, float] = (0.75, 0.25),
                            cyl_r: float = 0.05, steps: int = 500) -> Scene:
    """Water column plus air filling the rest of a closed-top box, with an
    inclined ramp and a vertical cylinder obstacle.

    Water (rho0 = 1000, continuity density) occupies x < column[0],
    z < column[2]; air (rho0 = 1, summation density, penalty on) fills every
    other site inside the tank that is outside the obstacles.  The ramp is
    the half space below the plane through (ramp_x0, z = 0) rising at
    ``ramp_deg`` towards +x; the cylinder is vertical at ``cyl_xy``.  Obstacle
    wall particles are the lattice sites with -layers*dp < sdf <= 0.  The box
    also has a roof (air must be contained).
    """
    ntx, nty, ntz = (_count(v, dp) for v in tank)
    ncx, ncz = _count(column[0], dp), _count(column[2], dp)
    h = 1.3 * dp
    H = ncz * dp
    inner = lattice((ntx, nty, ntz), dp)
    tan = math.tan(math.radians(ramp_deg))
    cosr = math.cos(math.radians(ramp_deg))

    def sdf_obstacles(p: np.ndarray) -> np.ndarray:
        # signed distance, negative inside solid
        ramp = (p[:, 2] - tan * (p[:, 0] - ramp_x0)) * cosr
        cyl = np.hypot(p[:, 0] - cyl_xy[0], p[:, 1] - cyl_xy[1]) - cyl_r
        return np.minimum(ramp, cyl)

    s = sdf_obstacles(inner)
    fluid_mask = s > 0.0
    obstacle_wall = inner[(s <= 0.0) & (s > -layers * dp)]
    fluid = inner[fluid_mask]
    water = (fluid[:, 0] < ncx * dp) & (fluid[:, 2] < H)
    phase = np.where(water, 0, 1).astype(np.int32)
    # closed box: walls on all six faces
    kx = np.arange(-layers, ntx + layers)
    ky = np.arange(-layers, nty + layers)
    kz = np.arange(-layers, ntz + layers)
    z, y, x = np.meshgrid(kz, ky, kx, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    inside = ((x >= 0) & (x < ntx) & (y >= 0) & (y < nty)
              & (z >= 0) & (z < ntz))
    box = (np.stack([x[~inside], y[~inside], z[~inside]], axis=1)
           .astype(np.float64) + 0.5) * dp
    wall = np.concatenate([box, obstacle_wall], axis=0)
    lo, hi = _domain(wall, fluid, 2 * h, 0.0, dp)
    c0 = 10.0 * math.sqrt(G * H)
    return Scene(
        name=(f"two_phase_ramp_cylinder_{tank[0]:g}x{tank[1]:g}x{tank[2]:g}"
              f"_dp{dp:g}"),
        dp=dp, h=h, c0=c0, g=(0.0, 0.0, -G), lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="linear", density="continuity",
                      reinit="free_surface", penalty=False, z_top=H),
                Phase(rho0=1.0, eos="linear", density="summation",
                      reinit="internal", penalty=True, z_top=ntz * dp)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid), fluid_phase=phase,
        wall_pos=wall, reinit_every=1, steps=steps)


def two_phase_still_tank(n: Tuple[int, int] = (12, 6), dp: float = 0.01,
                         water_layers: int = 6, air_layers: int = 6,
                         layers: int = 3) -> Scene:
    """Closed box with water below and air above, both at rest (a 3-D,
    thin-box stand-in for the paper's two-phase hydrostatic tank)."""
    nx, ny = n
    nz = water_layers + air_layers
    h = 1.3 * dp
    H = water_layers * dp
    fluid = lattice((nx, ny, nz), dp)
    phase = np.where(fluid[:, 2] < H, 0, 1).astype(np.int32)
    kx = np.arange(-layers, nx + layers)
    ky = np.arange(-layers, ny + layers)
    kz = np.arange(-layers, nz + layers)
    z, y, x = np.meshgrid(kz, ky, kx, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    inside = ((x >= 0) & (x < nx) & (y >= 0) & (y < ny) & (z >= 0) & (z < nz))
    wall = (np.stack([x[~inside], y[~inside], z[~inside]], axis=1)
            .astype(np.float64) + 0.5) * dp
    lo, hi = _domain(wall, fluid, 2 * h, 0.0, dp)
    return Scene(
        name=f"two_phase_still_tank_{nx}x{ny}x{nz}_dp{dp:g}", dp=dp, h=h,
        c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G), lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="linear", density="continuity",
                      reinit="free_surface", penalty=False, z_top=H),
                Phase(rho0=1.0, eos="linear", density="summation",
                      reinit="internal", penalty=True, z_top=nz * dp)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid), fluid_phase=phase,
        wall_pos=wall, reinit_every=1, steps=100)


def periodic_box(m: Tuple[int, int, int] = (1, 1, 1), dp: float = 0.01, jitter: float = 0.0,
                 vel_scale: float = 0.0, rho_jitter: float = 0.0, seed: int = 20211006,
                 eos: str = "linear", mu: float = 0.0) -> Scene:
    """A fluid-only box periodic along all three axes, filled with a lattice
    of spacing dp (optionally jittered by +-jitter dp, with random velocities
    of scale vel_scale and density excesses of relative scale rho_jitter), no
    walls, g = 0.  With h = 1.3 dp a period must be a whole number of 2h
    cells and of dp: 13 m particles = 5 m cells along each axis."""
    rng = np.random.default_rng(seed)
    n = tuple(13 * k for k in m)
    L = tuple(v * dp for v in n)
    fluid = lattice(n, dp)
    if jitter:
        fluid = fluid + rng.uniform(-jitter, jitter, fluid.shape) * dp
    vel = rng.normal(size=fluid.shape) * vel_scale if vel_scale else np.zeros_like(fluid)
    rho = 1000.0 * (1.0 + rho_jitter * rng.uniform(-1.0, 1.0, len(fluid)))
    return Scene(name=f"periodic_box_{n[0]}x{n[1]}x{n[2]}_dp{dp:g}", dp=dp, h=1.3 * dp, c0=10.0,
                 g=(0.0, 0.0, 0.0), lo=(0.0, 0.0, 0.0), hi=L,
                 phases=[Phase(rho0=1000.0, eos=eos, mu=mu, z_top=0.0)],
                 fluid_pos=fluid, fluid_vel=vel, fluid_phase=np.zeros(len(fluid), np.int32),
                 wall_pos=np.zeros((0, 3)), periodic=(1, 1, 1), reinit_every=0, rho_init=rho)


def periodic_channel(m: Tuple[int, int] = (1, 1), nz: int = 10, dp: float = 0.01, layers: int = 3,
                     dim: int = 3, eos: str = "tait") -> Scene:
    """Water at rest between a floor and a roof of wall particles, periodic
    along x (and y in 3-D): 13 m_x x 13 m_y x nz particles (13 m_x x nz in
    the 2-D form, in the plane y = 0), g = -9.81 z, hydrostatic density; the
    walls span the whole period."""
    nx = 13 * m[0]
    ny = 13 * m[1] if dim == 3 else 1
    Lx, Ly = nx * dp, ny * dp
    h = 1.3 * dp
    H = nz * dp
    if dim == 3:
        fluid = lattice((nx, ny, nz), dp)
        wl = lattice((nx, ny, layers), dp, origin=(0.0, 0.0, -layers * dp))
        wu = lattice((nx, ny, layers), dp, origin=(0.0, 0.0, H))
        lo = (0.0, 0.0, -layers * dp - 2 * h)
        hi = (Lx, Ly, H + layers * dp + 2 * h)
        per = (1, 1, 0)
    else:
        fluid = lattice2d((nx, nz), dp)
        wl = lattice2d((nx, layers), dp, origin=(0.0, -layers * dp))
        wu = lattice2d((nx, layers), dp, origin=(0.0, H))
        lo = (0.0, -2 * h, -layers * dp - 2 * h)
        hi = (Lx, 2 * h, H + layers * dp + 2 * h)
        per = (1, 0, 0)
    wall = np.concatenate([wl, wu])
    return Scene(name=f"periodic_channel_{nx}x{ny}x{nz}_dp{dp:g}_{dim}d", dp=dp, h=h,
                 c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G), lo=lo, hi=hi,
                 phases=[Phase(rho0=1000.0, eos=eos, z_top=H)], fluid_pos=fluid,
                 fluid_vel=np.zeros_like(fluid), fluid_phase=np.zeros(len(fluid), np.int32),
                 wall_pos=wall, periodic=per, reinit_every=1, dim=dim)


def jittered_blob(n: Tuple[int, int, int] = (16, 16, 16), dp: float = 0.01,
                  jitter: float = 0.05, vel_scale: float = 0.1,
                  rho_jitter: float = 0.0, seed: int = SEED_JITTER,
                  margin_cells: int = 4, eos: str = "tait") -> Scene:
    """Free fluid blob, no walls, no gravity: lattice sites moved by a
    uniform random jitter of +-jitter*dp, with random velocities of scale
    ``vel_scale`` (m/s).  Used for conservation checks."""
    rng = np.random.default_rng(seed)
    h = 1.3 * dp
    pos = lattice(n, dp)
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) * dp
    vel = rng.normal(0.0, vel_scale, size=pos.shape)
    lo = tuple(float(v) for v in (pos.min(axis=0) - margin_cells * 2 * h))
    hi = tuple(float(v) for v in (pos.max(axis=0) + margin_cells * 2 * h))
    sc = Scene(
        name=f"jittered_blob_{n[0]}x{n[1]}x{n[2]}_dp{dp:g}", dp=dp, h=h,
        c0=10.0, g=(0.0, 0.0, 0.0), lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos=eos, reinit="none",
                      z_top=float(pos[:, 2].max()))],
        fluid_pos=pos, fluid_vel=vel,
        fluid_phase=np.zeros(pos.shape[0], np.int32),
        wall_pos=np.zeros((0, 3)), reinit_every=0)
    if rho_jitter > 0.0:
        sc.rho_init = 1000.0 * (1.0 + rng.uniform(-rho_jitter, rho_jitter,
                                                  size=pos.shape[0]))
    return sc


# ------------------------------------------------------------------ 2-D
def lattice2d(n: Tuple[int, int], dp: float,
              origin: Tuple[float, float] = (0.0, 0.0)) -> np.ndarray:
    """(k + 1/2) dp sites of an nx x nz block in the plane y = 0."""
    nx, nz = n
    z, x = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    pts = np.stack([(x.ravel() + 0.5) * dp + origin[0], np.zeros(x.size),
                    (z.ravel() + 0.5) * dp + origin[1]], axis=1)
    return pts.astype(np.float64)


def box_walls2d(inner: Tuple[int, int], dp: float, layers: int = 3, roof: bool = True) -> np.ndarray:
    """Wall dummy particles filling ``layers`` lattice layers outside an
    inner box of nx x nz sites (floor and side walls, and a roof if asked)."""
    nx, nz = inner
    top = nz + layers if roof else nz
    kx = np.arange(-layers, nx + layers)
    kz = np.arange(-layers, top)
    z, x = np.meshgrid(kz, kx, indexing="ij")
    x, z = x.ravel(), z.ravel()
    inside = (x >= 0) & (x < nx) & (z >= 0) & ((z < nz) if roof else True)
    pts = np.stack([(x[~inside] + 0.5) * dp, np.zeros((~inside).sum()), (z[~inside] + 0.5) * dp], axis=1)
    return pts.astype(np.float64)


def _domain2d(wall: np.ndarray, fluid: np.ndarray, cell: float, head: float, dp: float):
    allp = np.concatenate([wall, fluid], axis=0)
    lo = (float(allp[:, 0].min() - cell - 0.1 * dp), -0.5 * cell,
          float(allp[:, 2].min() - cell - 0.1 * dp))
    hi = (float(allp[:, 0].max() + cell), 0.5 * cell, float(allp[:, 2].max() + cell + head))
    return lo, hi


def two_phase_hydrostatic_tank_2d(dx: float = 0.01, L: float = 1.0, H: float = 0.5,
                                  layers: int = 3) -> Scene:
    """The 2-D two-phase hydrostatic tank of Sec. 4.1: a closed tank of length
    L = 2H = 1 m and height 2H, water (rho0 = 1000) in the lower half, air
    (rho0 = 1) in the upper half, both at rest; particle spacing dx (the
    paper uses 0.01, 0.005, 0.0025, 0.00125 m).  Both fluids inviscid, linear
    EOS with one c0 = 10 sqrt(g H); air with summation density and the
    penalty force, as in the 3-D two-phase case."""
    nx, nz = _count(L, dx), _count(2 * H, dx)
    h = 1.3 * dx
    fluid = lattice2d((nx, nz), dx)
    phase = np.where(fluid[:, 2] < H, 0, 1).astype(np.int32)
    wall = box_walls2d((nx, nz), dx, layers, roof=True)
    lo, hi = _domain2d(wall, fluid, 2 * h, 0.0, dx)
    return Scene(
        name=f"two_phase_hydrostatic_tank_2d_dx{dx:g}", dp=dx, h=h,
        c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G), lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="linear", density="continuity",
                      reinit="free_surface", penalty=False, z_top=H),
                Phase(rho0=1.0, eos="linear", density="summation",
                      reinit="internal", penalty=True, z_top=2 * H)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid), fluid_phase=phase,
        wall_pos=wall, reinit_every=1, steps=1, dim=2)


def sloshing_tank_2d(dx: float = 0.01, L: float = 1.3, D: float = 0.9, H: float = 0.18,
                     layers: int = 3, air_penalty: bool = True) -> Scene:
    """The two-phase sloshing tank of Sec. 4.2 in the x-z plane: a closed tank
    of width L = 1.3 m and height D = 0.9 m, water (rho0 = 1000) to H = 0.18 m,
    air (rho0 = 1) above, at rest; the paper drives it with x = A0 sin(2 pi f0
    t), A0 = 0.1 m, f0 = 0.496 Hz (sph_set_excitation).  Linear EOS with one
    c0 = 10 sqrt(g H); air with summation density and, unless turned off, the
    penalty force of Eq. (SPH_penaltyMethodTerm)."""
    nx, nz = _count(L, dx), _count(D, dx)
    h = 1.3 * dx
    fluid = lattice2d((nx, nz), dx)
    phase = np.where(fluid[:, 2] < H, 0, 1).astype(np.int32)
    wall = box_walls2d((nx, nz), dx, layers, roof=True)
    lo, hi = _domain2d(wall, fluid, 2 * h, 0.0, dx)
    return Scene(
        name=f"sloshing_tank_2d_dx{dx:g}", dp=dx, h=h, c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G),
        lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="linear", density="continuity", reinit="free_surface",
                      penalty=False, z_top=H),
                Phase(rho0=1.0, eos="linear", density="summation", reinit="internal",
                      penalty=air_penalty, z_top=D)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid), fluid_phase=phase, wall_pos=wall,
        reinit_every=1, steps=1, dim=2)


def dam_break_2d(tank: Tuple[float, float] = (0.4, 0.3), column: Tuple[float, float] = (0.15, 0.15),
                 dx: float = 0.005, layers: int = 3, penalty: bool = True, reinit_every: int = 20) -> Scene:
    """A 2-D dam break in the x-z plane: a water column at x = 0 in an open
    tank (Tait EOS, penalty on, reinitialisation every 20 steps)."""
    ntx, ntz = _count(tank[0], dx), _count(tank[1], dx)
    ncx, ncz = _count(column[0], dx), _count(column[1], dx)
    h = 1.3 * dx
    H = ncz * dx
    fluid = lattice2d((ncx, ncz), dx)
    wall = box_walls2d((ntx, ntz), dx, layers, roof=False)
    lo, hi = _domain2d(wall, fluid, 2 * h, 0.25 * tank[1], dx)
    return Scene(
        name=f"dam_break_2d_{tank[0]:g}x{tank[1]:g}_dx{dx:g}", dp=dx, h=h,
        c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G), lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="tait", penalty=penalty, z_top=H)],
        fluid_pos=fluid, fluid_vel=np.zeros_like(fluid),
        fluid_phase=np.zeros(fluid.shape[0], np.int32), wall_pos=wall,
        reinit_every=reinit_every, steps=1, dim=2)


def perturbed(sc: Scene, jitter: float = 0.3, shift: Tuple[float, float, float] = (0.0, 0.0, 0.0),
              vel_scale: float = 0.0, mu: Optional[float] = None, seed: int = SEED_JITTER,
              reinit_every: Optional[int] = None) -> Scene:
    """A copy of a scene with its fluid moved by ``shift`` (in units of dp)
    plus a uniform random jitter of +-jitter*dp per coordinate, random normal
    velocities of scale ``vel_scale`` (m/s), and optionally another viscosity
    or reinitialisation period.  Moving the fluid towards the walls brings
    particles within dp/2 of the first wall layer, where the penalty force is
    active.  Used by the adjoint checks, which need every term of the step to
    matter."""
    rng = np.random.default_rng(seed)
    pos = (sc.fluid_pos + np.asarray(shift, np.float64) * sc.dp
           + rng.uniform(-jitter, jitter, size=sc.fluid_pos.shape) * sc.dp)
    vel = rng.normal(0.0, 1.0, size=pos.shape) * vel_scale
    phases = [dataclasses.replace(ph, mu=ph.mu if mu is None else mu) for ph in sc.phases]
    return dataclasses.replace(
        sc, name=sc.name + f"_perturbed{seed}", fluid_pos=pos, fluid_vel=vel, phases=phases,
        reinit_every=sc.reinit_every if reinit_every is None else reinit_every)


def compressed_clump(n: Tuple[int, int, int] = (12, 12, 10), dp: float = 0.01, spacing: float = 0.6,
                     layers: int = 3, margin: int = 6, vel_scale: float = 0.05, rho_jitter: float = 0.002,
                     mu: float = 0.0, seed: int = SEED_JITTER) -> Scene:
    """Fluid compressed to ``spacing`` dp (0.6: about 340 fluid neighbours
    within 2h = 2.6 dp, against about 80 on the lattice of spacing dp) resting
    on a floor of ``layers`` wall layers at the same spacing (about 180 wall
    neighbours for the lowest particles), reaching ``margin`` sites beyond the
    fluid on every side; the lowest fluid layer sits 0.45 dp above the top wall
    layer, inside the penalty's reach.  Particle masses stay rho0 dp^3 (the scene's dp), the
    density starts at rho0 (1 + rho_jitter U(-1, 1)), velocities are random
    normal of scale ``vel_scale``.  The state an impact compresses to: it
    makes the per-particle neighbour lists overflow, so the sweeps take their
    cell-scanning fallback.  No density reinitialisation: the number density is
    4.6 times the lattice's, which it would turn into a 4.6-fold density."""
    rng = np.random.default_rng(seed)
    s = spacing * dp
    h = 1.3 * dp
    fluid = lattice(n, s, origin=(0.0, 0.0, -0.25 * s))
    wall = lattice((n[0] + 2 * margin, n[1] + 2 * margin, layers), s,
                   origin=(-margin * s, -margin * s, -layers * s))
    H = n[2] * s
    lo, hi = _domain(wall, fluid, 2 * h, 2 * h, dp)
    rho = 1000.0 * (1.0 + rho_jitter * rng.uniform(-1.0, 1.0, fluid.shape[0]))
    vel = rng.normal(0.0, 1.0, size=fluid.shape) * vel_scale
    return Scene(
        name=f"compressed_clump_{n[0]}x{n[1]}x{n[2]}_s{spacing:g}dp", dp=dp, h=h,
        c0=10.0 * math.sqrt(G * H), g=(0.0, 0.0, -G), lo=lo, hi=hi,
        phases=[Phase(rho0=1000.0, eos="tait", penalty=True, mu=mu, z_top=H)],
        fluid_pos=fluid, fluid_vel=vel, fluid_phase=np.zeros(fluid.shape[0], np.int32),
        wall_pos=wall, reinit_every=0, steps=1, rho_init=rho)


def random_points(n: int, box: Tuple[float, float, float], seed: int,
                  dp: float = 0.01) -> np.ndarray:
    """n uniform random points in [0, box) (for neighbour-search checks)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(n, 3)) * np.asarray(box)


def standard(name: str) -> Scene:
    """The workloads the benchmark and the parity tests are defined on."""
    if name == "still_water_8k":
        return still_water_tank()
    if name == "dam_break_80k":
        return dam_break()
    if name == "two_phase_ramp_cylinder":
        return two_phase_ramp_cylinder()
    if name == "dam_break_obstacle_123k":
        return dam_break_obstacle()
    if name == "dam_break_adjoint_189k":
        # probes behind the column: the far wall sees no water within 10 steps
        return dam_break(dp=0.0075, steps=10, n_probes=64, probe_wall="near")
    if name == "dam_break_10m":
        return dam_break(tank=(3.2, 1.0, 1.0), column=(1.2, 1.0, 0.55),
                         dp=0.004, steps=200)
    raise KeyError(name)
