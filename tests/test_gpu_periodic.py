"""Periodic axes on the GPU (sph_params.periodic) against the FP64 oracle:
cell keys, order and ranges bit-exact in a jittered periodic box at create
and after steps with particles crossing the faces; the state within the
step tolerances of the parity suite; total momentum conserved (plain FP64
form to 1e-11, FP32 to the rounding of its pair sums); the full-lattice
number density in a filled periodic box; a periodic channel with floor and
roof (3-D and 2-D) matching the oracle; sensors across a periodic face;
the refusals (fractional period, periodic y in 2-D)."""
import ctypes as C
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2110_02621_gb300 import build, scenes as S, sph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    sph.lib()


def rel_inf(g, r, floor=0.0):
    den = max(np.abs(r).max(), floor)
    return float(np.abs(g - r).max() / den) if den > 0 else float(np.abs(g).max())


def check_cells(sim, ref):
    g, o = sim.cells(), ref.cells()
    assert np.array_equal(g["dims"], o["dims"])
    assert np.array_equal(g["key_f"], o["key_f"])
    assert np.array_equal(g["start_f"], o["start_f"].astype(np.int32))
    assert np.array_equal(g["order_f"], o["order_f"].astype(np.int32))


def moving_box(m=(1, 1, 1)):
    return S.periodic_box(m=m, jitter=0.3, vel_scale=0.2, rho_jitter=0.003, mu=1e-3)


@pytest.mark.parametrize("precision", [sph.SPH_FP32, sph.SPH_FP64_PLAIN])
def test_periodic_box_parity_and_cells(precision):
    sc = moving_box(m=(2, 1, 1))
    ref = oracle.OracleSim(sc)
    sim = sph.Simulation(sc, precision=precision)
    check_cells(sim, ref)
    dt = 2e-4
    for _ in range(3):
        ref.step(20, dt)
        sim.step(20, dt)
        g, o = sim.state(), ref.fluid()
        L = np.array(sc.hi)
        dx = g["x"] - o["x"]
        dx -= L * np.round(dx / L)  # a particle on a face may sit on either side
        tol = 1e-3 if precision == sph.SPH_FP32 else 1e-9
        assert np.abs(dx).max() <= tol * sc.dp
        assert np.all(g["x"] >= 0.0) and np.all(g["x"] < L)
        assert rel_inf(g["rho"] - 1000.0, o["rho"] - 1000.0) <= (2e-3 if precision == sph.SPH_FP32 else 1e-9)
        assert rel_inf(g["a"], o["a"]) <= (2e-3 if precision == sph.SPH_FP32 else 1e-8)
    if precision == sph.SPH_FP64_PLAIN:
        check_cells(sim, ref)
    # particles crossed the faces
    assert (np.abs(sim.state()["x"] - sc.fluid_pos) > 0.5 * np.array(sc.hi)).any()
    assert sim.diagnostics()[7] == 0.0
    sim.close()


@pytest.mark.parametrize("precision, tol", [(sph.SPH_FP64_PLAIN, 1e-11), (sph.SPH_FP32, 1e-5)])
def test_periodic_box_conserves_momentum(precision, tol):
    """Pair antisymmetry: each particle's sum is gathered separately, so the
    pair terms cancel to the rounding of the arithmetic (FP64: 1e-11 of the
    momentum scale; FP32: measured 1e-7 per step)."""
    sc = moving_box()
    sim = sph.Simulation(sc, precision=precision)
    d0 = sim.diagnostics()
    scale = 1000.0 * sc.dp ** 3 * np.abs(sc.fluid_vel).sum()
    sim.step(100, 2e-4)
    d = sim.diagnostics()
    assert np.abs(d[1:4] - d0[1:4]).max() < tol * scale
    assert d[0] == d0[0]
    sim.close()


def test_filled_periodic_lattice_has_the_lattice_number_density():
    sc = S.periodic_box()
    rho = np.full(sc.n_fluid, 1000.0)
    sim = sph.Simulation(sc, rho=rho)
    sim.step(1, 1e-6)
    st = sim.state()
    s0 = oracle.lattice_sigma0(sc.dp, sc.h)
    assert np.abs(st["sigma"] / s0 - 1.0).max() < 2e-6
    assert np.abs(st["a"]).max() < 1e-3
    sim.close()


@pytest.mark.parametrize("dim", [3, 2])
def test_periodic_channel_parity(dim):
    sc = S.periodic_channel(dim=dim)
    ref = oracle.OracleSim(sc)
    sim = sph.Simulation(sc)
    gw, ow = sim.state(), ref.wall()
    assert np.allclose(gw["normal"], ow["normal"], atol=1e-6)
    dt = 1e-4
    ref.step(50, dt)
    sim.step(50, dt)
    g, o, ow = sim.state(), ref.fluid(), ref.wall()
    assert np.abs(g["x"] - o["x"]).max() <= 1e-3 * sc.dp
    assert rel_inf(g["a"], o["a"], 9.81) <= 2e-5 * 10
    assert rel_inf(g["pw"], ow["pw"]) <= 2e-4
    sim.close()


def test_sensors_across_a_periodic_face():
    sc = S.periodic_box()
    rho = np.full(sc.n_fluid, 1003.0)
    ref = oracle.OracleSim(sc, rho=rho)
    sim = sph.Simulation(sc, rho=rho)
    L = np.array(sc.hi)
    pts = np.array([[0.0, 0.0, 0.0], [L[0] - 1e-4, 0.5 * L[1], 0.2 * L[2]], [0.5 * L[0], -0.01, 1.5 * L[2]]])
    pr, wr = ref.probe_pressure(pts)
    pg, wg = sim.probe_pressure(pts)
    assert np.abs(wg - wr).max() < 1e-6
    assert np.abs(wr - wr[0]).max() < 0.02 and wr.min() > 0.9  # a full support everywhere
    assert np.abs(pg - pr).max() < 1e-6 * abs(pr[0])
    sim.close()


def _params_status(sc):
    P = sph.make_params(sc, sph.SPH_FP32)
    x = np.ascontiguousarray(sc.fluid_pos)
    F = sph.sph_fluid(sc.n_fluid, x.ctypes.data_as(C.c_void_p), None, None, None)
    W = sph.sph_wall(0, None)
    st, ctx = sph.sph_create(P, F, W, None)
    if st == sph.SPH_OK:
        sph.sph_destroy(ctx)
    return st


def test_periodic_refusals():
    sc = S.periodic_box()
    assert _params_status(sc) == sph.SPH_OK
    bad = dataclasses.replace(sc, hi=(sc.hi[0] + 0.3 * sc.dp, sc.hi[1], sc.hi[2]))
    assert _params_status(bad) == sph.SPH_ERR_ARG
    two = S.periodic_channel(dim=2)
    assert _params_status(dataclasses.replace(two, periodic=(1, 1, 0))) == sph.SPH_ERR_ARG
    sim = sph.Simulation(moving_box())
    assert sph.sph_tape(sim.ctx, 1, 1e-4)[0] == sph.SPH_OK  # the adjoint covers periodic runs
    sim.close()
