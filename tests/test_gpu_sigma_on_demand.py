"""The number density sigma of Sec. 2.5 is needed only by a step that
reinitialises the density; the momentum sweep of the steps before others
leaves it out and the state export or sph_reinit_density computes it on
demand (k_sigma).  Both routes must give the same bits.

Two runs of the same dam break differ only in reinit_every (8 and 20): both
reinitialise at step 0 and nowhere else in their first 8 steps, so their
states agree bit for bit, but after 8 steps the first run's last momentum
sweep produced sigma (its step 8 reinitialises) while the second's left it
out."""
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


@pytest.mark.parametrize("precision", [sph.SPH_FP32, sph.SPH_FP64_PLAIN], ids=["fp32", "fp64"])
def test_sigma_on_demand_equals_the_sweep(precision):
    sc = S.perturbed(S.dam_break(tank=(0.3, 0.12, 0.15), column=(0.1, 0.12, 0.08), dp=0.01),
                     jitter=0.2, vel_scale=0.3)
    out = {}
    for every in (8, 20):
        with sph.Simulation(dataclasses.replace(sc, reinit_every=every), precision=precision) as sim:
            sim.step(8, 1e-4)
            out[every] = sim.state()
    for k in ("x", "v", "rho", "p", "a", "sigma", "pw"):
        assert np.array_equal(out[8][k], out[20][k]), k
    # and sigma is the oracle's number density at the same state
    ref = oracle.OracleSim(dataclasses.replace(sc, reinit_every=20))
    ref.step(8, 1e-4)
    o = ref.fluid()
    tol = 1e-12 if precision == sph.SPH_FP64_PLAIN else 1e-5
    assert np.abs(out[20]["sigma"] - o["sigma"]).max() <= tol * np.abs(o["sigma"]).max()


def test_explicit_reinit_uses_the_current_sigma():
    """sph_reinit_density right after a step without sigma: the same state as
    after a step that produced it."""
    sc = S.perturbed(S.dam_break(tank=(0.3, 0.12, 0.15), column=(0.1, 0.12, 0.08), dp=0.01),
                     jitter=0.2, vel_scale=0.3)
    out = {}
    for every in (8, 20):
        with sph.Simulation(dataclasses.replace(sc, reinit_every=every)) as sim:
            sim.step(8, 1e-4)
            sim.reinit_density()
            out[every] = sim.state()
    for k in ("rho", "p", "sigma"):
        assert np.array_equal(out[8][k], out[20][k]), k
