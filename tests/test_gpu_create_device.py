"""sph_create_device: a context whose fluid state starts from device arrays
(Sec. 3: one upload, then device-resident state) equals the context
sph_create makes from the same values in host memory, bit for bit, after
create and after steps; device inputs that sph_create would refuse on the
host are refused by the device-side check, before any other use."""
import numpy as np
import pytest

from paper_2110_02621_gb300 import build, scenes as S, sph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    sph.lib()


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype)).cuda()


def _same_state(a, b):
    for k in ("x", "v", "rho", "p", "a", "pw", "rhow"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision", [sph.SPH_FP32, sph.SPH_FP64_PLAIN])
def test_device_create_equals_host_create(precision):
    sc = S.perturbed(S.dam_break(tank=(0.3, 0.12, 0.15), column=(0.1, 0.12, 0.08), dp=0.01),
                     jitter=0.2, vel_scale=0.2)
    rho = 1000.0 * (1.0 + 1e-3 * np.random.default_rng(3).uniform(-1, 1, sc.n_fluid))
    with sph.Simulation(sc, precision=precision, rho=rho) as host:
        x, v, r = _dev(sc.fluid_pos, np.float64), _dev(sc.fluid_vel, np.float64), _dev(rho, np.float64)
        dev = sph.Simulation.from_device(sc, x, v, r, precision=precision)
        del x, v, r  # the context keeps its own copies
        _same_state(host.state(), dev.state())
        host.step(5, 1e-4)
        dev.step(5, 1e-4)
        _same_state(host.state(), dev.state())
        dev.close()


def test_device_create_two_phases_and_hydrostatic_start():
    sc = S.two_phase_still_tank()
    with sph.Simulation(sc) as host:
        dev = sph.Simulation.from_device(sc, _dev(sc.fluid_pos, np.float64), _dev(sc.fluid_vel, np.float64),
                                         None, _dev(sc.fluid_phase, np.int32))
        _same_state(host.state(), dev.state())
        dev.close()


@pytest.mark.parametrize("bad", ["nan_x", "inf_v", "rho_zero", "phase"])
def test_device_create_refuses_bad_inputs(bad):
    sc = S.two_phase_still_tank()
    x, v = sc.fluid_pos.copy(), sc.fluid_vel.copy()
    rho = np.full(sc.n_fluid, 1000.0)
    ph = sc.fluid_phase.astype(np.int32).copy()
    k = sc.n_fluid // 2
    if bad == "nan_x":
        x[k, 1] = np.nan
    elif bad == "inf_v":
        v[k, 2] = np.inf
    elif bad == "rho_zero":
        rho[k] = 0.0
    else:
        ph[k] = 2
    with pytest.raises(sph.SphError) as e:
        sph.Simulation.from_device(sc, _dev(x, np.float64), _dev(v, np.float64), _dev(rho, np.float64),
                                   _dev(ph, np.int32))
    assert e.value.status == sph.SPH_ERR_ARG
