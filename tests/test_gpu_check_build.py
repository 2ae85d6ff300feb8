"""The index-checking debug build (build.build(check=True), -DSPH_CHECK).

In that build every index the kernels read from memory (neighbour-list
entries, cell keys, cell ranges, sort slots, the adjoint's permutations) is
checked before it addresses anything; an index out of range sets a bit of a
check word that the host turns into SPH_ERR_CUDA.  It stands in for a memory
checker.  These tests build it once and run the small parity scenes through
it: every run must end with a clear check word and give the same bits as the
normal build (the checks change nothing while indices are in range), and
the normal build's results agree with the oracle elsewhere.
"""
import numpy as np
import pytest

from paper_2110_02621_gb300 import build, scenes as S, sph

pytestmark = pytest.mark.gpu

DT = 1e-4


@pytest.fixture(scope="module")
def libs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    normal = build.build()
    checked = build.build(check=True)
    prev = sph.use_library(None)
    yield normal, checked
    sph.use_library(prev)


def run(path, scene, steps, precision, rho=None, backward=False):
    """State after `steps` fixed steps (and the adjoint of a taped run) with
    the library at `path`."""
    sph.use_library(path)
    sim = sph.Simulation(scene, precision=precision, rho=rho)
    try:
        if backward:
            sim.tape(steps, DT)
        else:
            sim.step(steps, DT)
        out = {"state": sim.state(), "cells": sim.cells(), "nb": sim.neighbors()}
        if backward:
            rng = np.random.default_rng(7)
            seed = {"x": rng.normal(size=(scene.n_fluid, 3)), "v": rng.normal(size=(scene.n_fluid, 3))}
            out["grad"] = sim.backward(seed)
        return out
    finally:
        sim.close()


def same(a, b):
    for k in ("x", "v", "rho", "p", "a", "pw"):
        assert np.array_equal(a["state"][k], b["state"][k]), k
    for k in ("key_f", "order_f", "start_f"):
        assert np.array_equal(a["cells"][k], b["cells"][k]), k
    for k in ("f_off", "f_ids", "w_off", "w_ids"):
        assert np.array_equal(a["nb"][k], b["nb"][k]), k
    if "grad" in a:
        for k in ("x", "v", "rho"):
            assert np.array_equal(a["grad"][k], b["grad"][k]), k


SCENES = {
    "still_water_8k": lambda: S.still_water_tank(),
    "dam_break_small": lambda: S.perturbed(S.dam_break(tank=(0.3, 0.12, 0.15), column=(0.1, 0.12, 0.08),
                                                       dp=0.01), jitter=0.2, vel_scale=0.3),
    "two_phase_still": lambda: S.two_phase_still_tank(),
    "periodic_box": lambda: S.periodic_box(jitter=0.3, vel_scale=0.3),
    "overflowing_clump": lambda: S.compressed_clump(),
}


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("precision", [sph.SPH_FP32, sph.SPH_FP64_PLAIN], ids=["fp32", "fp64"])
def test_checked_build_runs_clean_and_matches(libs, name, precision):
    normal, checked = libs
    sc = SCENES[name]()
    steps = 2 if name == "overflowing_clump" else 20  # the clump is far from equilibrium
    a = run(normal, sc, steps, precision)
    b = run(checked, sc, steps, precision)  # raises SphError(SPH_ERR_CUDA) on a failed check
    same(a, b)


def test_checked_build_adjoint(libs):
    normal, checked = libs
    sc = S.perturbed(S.dam_break(tank=(0.2, 0.1, 0.12), column=(0.08, 0.1, 0.06), dp=0.01),
                     jitter=0.3, shift=(-0.3, 0.0, -0.3), vel_scale=0.3, mu=0.05, reinit_every=2)
    a = run(normal, sc, 3, sph.SPH_FP64_PLAIN, backward=True)
    b = run(checked, sc, 3, sph.SPH_FP64_PLAIN, backward=True)
    same(a, b)
