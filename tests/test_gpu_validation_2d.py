"""The 2-D two-phase hydrostatic tank of Sec. 4.1 on the GPU (FP32 form):
water below, air above, both at rest, run for 10 s.

Checked: the potential energy at t = 0 is the paper's T_tot = 1226.25 J
(tests/golden/hydrostatic_tank_2d.json) plus the air's rho_a g L ((2H)^2 -
H^2)/2; mass is exactly conserved; the system comes to rest (E_kin(10 s) <
1e-4 T_tot); the total energy changes by less than 1.5 % of T_tot (measured
0.83-0.87 % at dx = 0.02, 0.01, 0.005; the paper reports 0.26 % with its own
sound speed); the water pressure stays within 2 % (relative L2) of the
hydrostatic profile rho_w g (H - z) + rho_a g H (measured 0.9-1.3 %); no
air particle sinks into the water."""
import json
import os

import numpy as np
import pytest

from paper_2110_02621_gb300 import build, scenes as S, sph

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hydrostatic_tank_2d.json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    sph.lib()


@pytest.mark.parametrize("dx", [0.02, 0.01])
def test_two_phase_hydrostatic_tank_2d(dx):
    ref = json.load(open(GOLDEN))
    L, H, g, rw = ref["L_m"], ref["H_m"], ref["g"], ref["rho_w"]
    ra = 1.0
    sc = S.two_phase_hydrostatic_tank_2d(dx=dx, L=L, H=H)
    with sph.Simulation(sc) as sim:
        d0 = sim.diagnostics()
        air_ep = ra * g * L * ((2 * H) ** 2 - H ** 2) / 2.0
        assert d0[5] == pytest.approx(ref["T_tot_J"] + air_ep, rel=1e-6)
        t = 0.0
        while t < 10.0:
            t += 200 * sim.step(200)
        st, d = sim.state(), sim.diagnostics()
    assert d[0] == d0[0]
    assert d[4] < 1e-4 * ref["T_tot_J"]
    assert abs((d[4] + d[5]) - (d0[4] + d0[5])) < 0.015 * ref["T_tot_J"]
    z, ph = st["x"][:, 2], sc.fluid_phase
    w = ph == 0
    p_a = rw * g * (H - z[w]) + ra * g * H
    l2 = np.sqrt(((st["p"][w] - p_a) ** 2).sum() / (p_a ** 2).sum())
    assert l2 < 0.02, l2
    assert not np.any((ph == 1) & (z < H - 5 * dx))
    assert np.all(np.abs(st["x"][:, 0] - 0.5 * L) < 0.5 * L + 0.5 * dx)
