"""CUDA sensors and wave gauges (sph_probe_pressure, sph_gauge_height; the
sensors P_i and gauges H_i of Sec. 4.3) against the FP64 oracle.

Tolerances:
  * on the initial state, shared by both sides up to the FP32 rounding of
    the stored state (offsets, density excess, pressure; 2^-24 relative):
    sensors within 1e-6 of rho0 g H (pressure) and 1e-6 (kernel sum), gauges
    within 1e-6 dx -- the linear interpolation makes the height continuous in
    phi, so a sample that rounds to the other side of 1/2 moves it by rounding
    only;
  * the plain FP64 form: 1e-9 relative;
  * after steps, the sensors sample states that differ by the FP32 rounding
    of 100 steps: 1e-5 of rho0 g H for the pressure and 1e-5 for the kernel
    sum (measured 2.5e-7 and 1.2e-7 after 100 steps, 8e-7 and 1.2e-7 after
    200, dam break with an obstacle at dx = 0.032 m), 1e-4 dx for the gauges
    (measured 1.4e-6 dx); the FP64 form within 1e-11 (measured 2e-14).
"""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
from paper_2110_02621_gb300 import build, scenes as S, sph

pytestmark = pytest.mark.gpu
G = 9.81


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    sph.lib()


def obstacle_small():
    return S.dam_break_obstacle(dp=0.032)


def sensor_points(sc, n_extra=40, seed=3):
    """The scene's sensors plus seeded points spread over the fluid's box and
    a margin of 3h around it (dry points, faces and edges included)."""
    rng = np.random.default_rng(seed)
    lo = sc.fluid_pos.min(0) - 3 * sc.h
    hi = sc.fluid_pos.max(0) + 3 * sc.h
    pts = lo + (hi - lo) * rng.random((n_extra, 3))
    if sc.dim == 2:
        pts[:, 1] = sc.fluid_pos[0, 1]
    base = sc.sensors if sc.sensors is not None else np.zeros((0, 3))
    return np.concatenate([base, pts])


def gauge_lines(sc, n_extra=12, seed=5):
    rng = np.random.default_rng(seed)
    lo, hi = sc.fluid_pos.min(0), sc.fluid_pos.max(0)
    xy = lo[:2] + (hi[:2] - lo[:2]) * rng.random((n_extra, 2))
    if sc.dim == 2:
        xy[:, 1] = sc.fluid_pos[0, 1]
    z_top = float(sc.hi[2]) - 0.01
    lines = np.column_stack([xy, np.full(n_extra, float(sc.lo[2]) + 0.001), np.full(n_extra, z_top)])
    base = sc.gauges if sc.gauges is not None else np.zeros((0, 4))
    return np.concatenate([base, lines])


def pressure_scale(sc):
    H = max(ph.z_top for ph in sc.phases)
    return max(ph.rho0 for ph in sc.phases) * G * H


SCENES_T0 = {
    "still_water_8k": lambda: S.still_water_tank(),
    "obstacle_dp0.032": obstacle_small,
    "two_phase_tank_2d": lambda: S.two_phase_hydrostatic_tank_2d(dx=0.02),
    "two_phase_ramp_cylinder": lambda: S.two_phase_ramp_cylinder(dp=0.01),
}


@pytest.mark.parametrize("name", list(SCENES_T0))
@pytest.mark.parametrize("precision", [sph.SPH_FP32, sph.SPH_FP64_PLAIN])
def test_sensors_and_gauges_on_the_initial_state(name, precision):
    sc = SCENES_T0[name]()
    pts, lines = sensor_points(sc), gauge_lines(sc)
    ref = oracle.OracleSim(sc)
    sim = sph.Simulation(sc, precision=precision)
    pr, wr = ref.probe_pressure(pts)
    pg, wg = sim.probe_pressure(pts)
    dz = 0.25 * sc.dp
    Hr, Hg = ref.gauge_height(lines, dz), sim.gauge_height(lines, dz)
    tol = 1e-6 if precision == sph.SPH_FP32 else 1e-9
    ps = pressure_scale(sc)
    assert np.abs(wg - wr).max() <= tol
    assert np.abs(pg - pr).max() <= tol * ps
    assert np.abs(Hg - Hr).max() <= tol * sc.dp
    assert np.array_equal(wg == 0.0, wr == 0.0)  # dry points agree exactly
    # the sample spans wet, dry and partial points
    assert (wr > 0.9).any() and (wr == 0.0).any() and ((wr > 0.1) & (wr < 0.9)).any()
    sim.close()
    ref.close()


def test_sensors_after_steps_fp32_and_fp64():
    """Obstacle dam break at dx = 0.032 m, 100 steps of fixed dt: both forms
    against the oracle's run."""
    sc = obstacle_small()
    pts, lines = sensor_points(sc), gauge_lines(sc)
    dt = 2e-4
    ref = oracle.OracleSim(sc)
    ref.step(100, dt)
    pr, wr = ref.probe_pressure(pts)
    Hr = ref.gauge_height(lines, 0.25 * sc.dp)
    ps = pressure_scale(sc)
    for precision, tp, tH in ((sph.SPH_FP32, 1e-5, 1e-4), (sph.SPH_FP64_PLAIN, 1e-11, 1e-11)):
        sim = sph.Simulation(sc, precision=precision)
        sim.step(100, dt)
        pg, wg = sim.probe_pressure(pts)
        Hg = sim.gauge_height(lines, 0.25 * sc.dp)
        assert np.abs(pg - pr).max() <= tp * ps, precision
        assert np.abs(wg - wr).max() <= tp, precision
        assert np.abs(Hg - Hr).max() <= tH * sc.dp, precision
        sim.close()


def test_ragged_counts_and_many_chunks():
    """1, 31, 33 and 1000 sensors (warps across blocks); gauges of 1 sample,
    127, 128, 129 and ~5000 samples (several chunks of 128)."""
    sc = S.still_water_tank((20, 20, 20), dp=0.01)
    ref = oracle.OracleSim(sc)
    sim = sph.Simulation(sc)
    allp = sensor_points(sc, n_extra=1000, seed=11)
    for n in (1, 31, 33, 1000):
        pr, wr = ref.probe_pressure(allp[:n])
        pg, wg = sim.probe_pressure(allp[:n])
        assert np.abs(pg - pr).max() <= 1e-6 * pressure_scale(sc)
        assert np.abs(wg - wr).max() <= 1e-6
    dz = 0.0025
    lines = []
    for K in (0, 126, 127, 128, 5000):
        top = 0.19 + 0.00031 * K  # the top sample above or below the surface
        lines.append([0.1, 0.1, top - K * dz, top])
    lines = np.array(lines)
    Hr, Hg = ref.gauge_height(lines, dz), sim.gauge_height(lines, dz)
    assert np.abs(Hg - Hr).max() <= 1e-6 * sc.dp
    sim.close()


def test_points_outside_the_grid_and_empty_calls():
    sc = S.still_water_tank()
    sim = sph.Simulation(sc)
    far = np.array([[1e30, 0.0, 0.0], [-1e30, -1e30, 1e30], [0.1, 0.1, 5.0], [-3.0, 0.1, 0.1]])
    p, w = sim.probe_pressure(far)
    assert np.all(p == 0.0) and np.all(w == 0.0)
    H = sim.gauge_height(np.array([[1e20, 0.0, 0.0, 1.0], [0.1, 0.1, 0.5, 0.6]]), 0.01)
    assert np.array_equal(H, [0.0, 0.5])  # dry lines: z_lo
    assert sph.sph_probe_pressure(sim.ctx, None, 0, None, None) == sph.SPH_OK
    assert sph.sph_gauge_height(sim.ctx, None, 0, 0.01, None) == sph.SPH_OK
    sim.close()


def _raw(a):
    return np.ascontiguousarray(a, np.float64).ctypes.data_as(C.c_void_p)


def test_invalid_arguments_are_rejected():
    sc = S.still_water_tank()
    sim = sph.Simulation(sc)
    ok = np.array([[0.1, 0.1, 0.1]])
    out = np.zeros(4)
    bad = np.array([[0.1, np.nan, 0.1]])
    assert sph.sph_probe_pressure(sim.ctx, _raw(bad), 1, _raw(out), None) == sph.SPH_ERR_ARG
    assert sph.sph_probe_pressure(sim.ctx, _raw(ok), -1, _raw(out), None) == sph.SPH_ERR_ARG
    assert sph.sph_probe_pressure(sim.ctx, None, 1, _raw(out), None) == sph.SPH_ERR_ARG
    assert sph.sph_probe_pressure(sim.ctx, _raw(ok), 1, _raw(out), None, 7) == sph.SPH_ERR_ARG
    line = np.array([[0.1, 0.1, 0.0, 0.3]])
    inverted = np.array([[0.1, 0.1, 0.3, 0.0]])
    inf = np.array([[0.1, 0.1, 0.0, np.inf]])
    for dz in (0.0, -1.0, np.nan, np.inf):
        assert sph.sph_gauge_height(sim.ctx, _raw(line), 1, dz, _raw(out)) == sph.SPH_ERR_ARG
    assert sph.sph_gauge_height(sim.ctx, _raw(inverted), 1, 0.01, _raw(out)) == sph.SPH_ERR_ARG
    assert sph.sph_gauge_height(sim.ctx, _raw(inf), 1, 0.01, _raw(out)) == sph.SPH_ERR_ARG
    many = 0.3 / sph.SPH_GAUGE_MAX_SAMPLES
    assert sph.sph_gauge_height(sim.ctx, _raw(line), 1, many, _raw(out)) == sph.SPH_ERR_ARG
    assert sph.sph_gauge_height(sim.ctx, _raw(line), 1, 0.01, None) == sph.SPH_ERR_ARG
    # the context stays usable
    p, _ = sim.probe_pressure(ok)
    assert p[0] > 0.0
    sim.close()


def test_device_buffers_and_a_recorded_series_match_the_host_calls():
    """DEVICE pointers: enqueued between sph_step_async calls into one device
    buffer per step (a sensor time series), then compared bit for bit with
    host calls after synchronous steps of the same run; an invalid line in
    device memory yields NaN."""
    torch = pytest.importorskip("torch")
    sc = obstacle_small()
    pts, lines = sc.sensors, np.concatenate([sc.gauges, [[0.5, 0.5, 0.3, 0.1]]])
    nsteps, dt = 6, 2e-4
    dev = torch.device("cuda")
    tp = torch.from_numpy(pts).to(dev)
    tl = torch.from_numpy(lines).to(dev)
    series_p = torch.zeros((nsteps, len(pts)), dtype=torch.float64, device=dev)
    series_w = torch.zeros((nsteps, len(pts)), dtype=torch.float64, device=dev)
    series_H = torch.zeros((nsteps, len(lines)), dtype=torch.float64, device=dev)
    a = sph.Simulation(sc)
    for k in range(nsteps):
        assert sph.sph_step_async(a.ctx, 1, dt) == sph.SPH_OK
        assert sph.sph_probe_pressure(a.ctx, tp.data_ptr(), len(pts), series_p[k].data_ptr(),
                                      series_w[k].data_ptr(), sph.SPH_DEVICE) == sph.SPH_OK
        assert sph.sph_gauge_height(a.ctx, tl.data_ptr(), len(lines), 0.008, series_H[k].data_ptr(),
                                    sph.SPH_DEVICE) == sph.SPH_OK
    st, _ = sph.sph_sync(a.ctx)
    assert st == sph.SPH_OK
    b = sph.Simulation(sc)
    for k in range(nsteps):
        b.step(1, dt)
        p, w = b.probe_pressure(pts)
        H = b.gauge_height(lines[:-1], 0.008)
        assert np.array_equal(series_p[k].cpu().numpy(), p)
        assert np.array_equal(series_w[k].cpu().numpy(), w)
        assert np.array_equal(series_H[k, :-1].cpu().numpy(), H)
        assert math.isnan(float(series_H[k, -1]))
    a.close()
    b.close()
