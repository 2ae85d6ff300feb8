"""The CUDA adjoint (sph_tape / sph_backward) against the FP64 reference
adjoint of oracle/adjoint.py and against central differences of the CUDA
forward, through the C ABI.

Tolerances:
  * the plain FP64 form: every gradient within 1e-8 of its infinity norm
    (the two adjoints differ only by rounding order);
  * the FP32 form: within 2e-3 of the infinity norm per field and 2e-3
    relative for the parameters.  The adjoint of an n-step run multiplies n
    step Jacobians; each FP32 pair sum carries the forward's relative error
    (2e-5 of the field scale, see test_gpu_parity) and the derivative terms
    (dF/dr, the limiter) are larger than the values by a factor of order
    2h/r ~ 10, so 3 steps allow ~1e-3;
  * central differences of the FP64 forward: 1e-6 relative.
The FP32 comparison does not seed p_w on walls whose fluid support at the
end is not empty but sums to less than 1e-2 W(0).  For a wall supported by
a single particle at the rim of its kernel, Eq. (wallPressure) gives
p_w = p_f + rho_f g.r_wf whatever W_wf, but its backward multiplies the
FP32 residual p_f + ... - p_w (zero in exact arithmetic) by
W'/W ~ 1/(1 - q/2), unbounded at the rim: the FP32 gradient of such a
wall's pressure is noise.  The FP64 comparisons seed every wall.
"""
import numpy as np
import pytest

import oracle
from oracle import adjoint as A
from paper_2110_02621_gb300 import build, scenes as S, sph

pytestmark = pytest.mark.gpu

DT = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    pytest.importorskip("scipy")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    sph.lib()


def adjoint_scene(mu=0.05, reinit_every=2, vel_scale=0.3):
    sc = S.dam_break(tank=(0.2, 0.1, 0.12), column=(0.08, 0.1, 0.06), dp=0.01)
    return S.perturbed(sc, jitter=0.3, shift=(-0.3, 0.0, -0.3), vel_scale=vel_scale, mu=mu,
                       reinit_every=reinit_every)


def reference(sc):
    ref = oracle.OracleSim(sc)
    return ref.fluid()["rho"].copy(), ref.wall()["normal"].copy(), ref.sigma0


def seeds(sc, rng):
    return {"x": rng.normal(size=(sc.n_fluid, 3)), "v": rng.normal(size=(sc.n_fluid, 3)),
            "rho": rng.normal(size=sc.n_fluid) * 1e-3, "pw": rng.normal(size=sc.n_wall) * 1e-3}


def rim_walls(sc, x, floor=1e-2):
    """Mask of the walls whose fluid support at positions x is not empty but
    sums to less than floor W(0) (Wendland C2 in units of W(0):
    (1 - q/2)^4 (2q + 1))."""
    from scipy.spatial import cKDTree
    h = sc.h
    out = np.zeros(sc.n_wall, bool)
    for w, fl in enumerate(cKDTree(x).query_ball_point(sc.wall_pos, 2 * h)):
        if fl:
            q = np.linalg.norm(x[fl] - sc.wall_pos[w], axis=1) / h
            out[w] = ((1 - q / 2) ** 4 * (2 * q + 1)).sum() < floor
    return out


def gpu_run(sc, rho0, nsteps, precision, seed=None):
    sim = sph.Simulation(sc, precision=precision, rho=rho0)
    sim.tape(nsteps, DT)
    st = sim.state()
    g = sim.backward(seed) if seed is not None else None
    return sim, st, g


def rel_inf(g, r):
    g, r = np.asarray(g, np.float64), np.asarray(r, np.float64)
    den = np.abs(r).max()
    return float(np.abs(g - r).max() / den) if den > 0 else float(np.abs(g).max())


def compare(g, o, tol_field, tol_param):
    for k in ("x", "v", "rho"):
        assert rel_inf(g[k], o[k]) <= tol_field, (k, rel_inf(g[k], o[k]))
    for k in ("c0", "gamma_p", "mu"):
        ref = float(o[k])
        assert abs(g[k] - ref) <= tol_param * max(abs(ref), 1e-12), (k, g[k], ref)


@pytest.mark.parametrize("nsteps", [0, 1, 3])
def test_adjoint_fp64_matches_reference(nsteps):
    sc = adjoint_scene()
    rho0, normals, sigma0 = reference(sc)
    seed = seeds(sc, np.random.default_rng(11 + nsteps))
    final, o, _ = A.vjp(sc, normals, sigma0, rho0, nsteps, DT, seed)
    sim, st, g = gpu_run(sc, rho0, nsteps, sph.SPH_FP64_PLAIN, seed)
    assert np.abs(st["x"] - final["x"]).max() < 1e-12
    assert rel_inf(st["pw"], final["pw"]) < 1e-10
    compare(g, o, 1e-8, 1e-8)
    if nsteps > 0:  # with no step the loss does not see a^0, where mu and gamma_p act
        assert abs(o["gamma_p"]) > 0 and abs(o["mu"]) > 0
    sim.close()


def test_adjoint_fp64_fast_flow_with_cell_changes():
    """2 m/s random velocities: particles change cells during the run (so the
    sorted order of each step differs) and the limiter saturates at c0."""
    sc = adjoint_scene(vel_scale=2.0)
    rho0, normals, sigma0 = reference(sc)
    seed = seeds(sc, np.random.default_rng(17))
    final, o, _ = A.vjp(sc, normals, sigma0, rho0, 4, DT, seed)
    sim, st, g = gpu_run(sc, rho0, 4, sph.SPH_FP64_PLAIN, seed)
    moved = np.floor((st["x"] - np.asarray(sc.lo)) / (2 * sc.h)) != np.floor(
        (sc.fluid_pos - np.asarray(sc.lo)) / (2 * sc.h))
    assert moved.any(axis=1).sum() > 10
    compare(g, o, 1e-8, 1e-8)
    sim.close()


def periodic_adjoint_scenes():
    box = S.periodic_box(jitter=0.3, vel_scale=0.3, rho_jitter=0.003, mu=0.05)
    chan = S.perturbed(S.periodic_channel(nz=6), jitter=0.3, shift=(0.0, 0.0, -0.3), vel_scale=0.3, mu=0.05,
                       reinit_every=2)
    return {"box": box, "channel": chan}


@pytest.mark.parametrize("name", ["box", "channel"])
def test_adjoint_with_periodic_axes_matches_reference(name):
    """A periodic box and a channel periodic along x and y: the CUDA adjoint
    (both forms, kept products and recompute alike) against the reference
    adjoint's nearest images."""
    sc = periodic_adjoint_scenes()[name]
    rho0, normals, sigma0 = reference(sc)
    seed = seeds(sc, np.random.default_rng(23))
    if sc.n_wall == 0:
        seed.pop("pw")
    final, o, _ = A.vjp(sc, normals, sigma0, rho0, 3, DT, seed)
    sim, st, g = gpu_run(sc, rho0, 3, sph.SPH_FP64_PLAIN, seed)
    compare(g, o, 1e-8, 1e-8)
    sim.close()
    sim = sph.Simulation(sc, precision=sph.SPH_FP64_PLAIN, rho=rho0)
    sim.tape_budget(0)
    sim.tape(3, DT)
    g0 = sim.backward(seed)
    for k in ("x", "v", "rho"):
        assert np.array_equal(g0[k], g[k]), k
    sim.close()
    _, _, g32 = gpu_run(sc, rho0, 3, sph.SPH_FP32, seed)
    compare(g32, o, 2e-3, 2e-3)


def test_adjoint_fp32_matches_reference():
    sc = adjoint_scene()
    rho0, normals, sigma0 = reference(sc)
    seed = seeds(sc, np.random.default_rng(5))
    final, _, _ = A.vjp(sc, normals, sigma0, rho0, 3, DT, seed)
    rim = rim_walls(sc, np.asarray(final["x"]))
    assert rim.sum() < 0.1 * sc.n_wall
    seed["pw"] = np.where(rim, 0.0, seed["pw"])
    _, o, _ = A.vjp(sc, normals, sigma0, rho0, 3, DT, seed)
    sim, _, g = gpu_run(sc, rho0, 3, sph.SPH_FP32, seed)
    compare(g, o, 2e-3, 2e-3)
    sim.close()


def test_adjoint_fp64_central_differences_of_the_cuda_forward():
    """Directional derivatives: L(theta + e d) - L(theta - e d) over 2e from
    the CUDA FP64 forward, against the CUDA adjoint."""
    sc = adjoint_scene()
    rho0, _, _ = reference(sc)
    rng = np.random.default_rng(21)
    seed = seeds(sc, rng)
    n = 3
    sim, _, g = gpu_run(sc, rho0, n, sph.SPH_FP64_PLAIN, seed)
    sim.close()

    def loss(s, r):
        q = sph.Simulation(s, precision=sph.SPH_FP64_PLAIN, rho=r)
        q.step(n, DT)
        st = q.state()
        q.close()
        return sum(float((st[k] * seed[k]).sum()) for k in ("x", "v", "rho", "pw"))

    import copy
    for name, eps in (("x", 1e-7), ("v", 1e-5), ("rho", 1e-2)):
        d = rng.normal(size=np.shape(g[name]))
        sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
        rp, rm = rho0, rho0
        if name == "x":
            sp.fluid_pos = sc.fluid_pos + eps * d
            sm.fluid_pos = sc.fluid_pos - eps * d
        elif name == "v":
            sp.fluid_vel = sc.fluid_vel + eps * d
            sm.fluid_vel = sc.fluid_vel - eps * d
        else:
            rp, rm = rho0 + eps * d, rho0 - eps * d
        fd = (loss(sp, rp) - loss(sm, rm)) / (2 * eps)
        ad = float((g[name] * d).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (name, fd, ad)
    for name, eps in (("c0", 1e-5 * sc.c0), ("gamma_p", 1e-3), ("mu", 1e-4)):
        sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
        if name == "c0":
            sp.c0 += eps
            sm.c0 -= eps
        elif name == "gamma_p":
            sp.gamma_p += eps
            sm.gamma_p -= eps
        else:
            sp.phases[0].mu += eps
            sm.phases[0].mu -= eps
        fd = (loss(sp, rho0) - loss(sm, rho0)) / (2 * eps)
        assert abs(fd - g[name]) <= 1e-6 * abs(g[name]), (name, fd, g[name])


def test_translation_invariance_on_gpu():
    sc = S.jittered_blob(n=(8, 8, 8), jitter=0.05, vel_scale=0.1)
    sc.phases[0].mu = 0.01
    sc.reinit_every = 2
    rho0 = oracle.OracleSim(sc).fluid()["rho"]
    rng = np.random.default_rng(3)
    seed = {"x": rng.normal(size=(sc.n_fluid, 3)), "v": rng.normal(size=(sc.n_fluid, 3))}
    sim, _, g = gpu_run(sc, rho0, 4, sph.SPH_FP64_PLAIN, seed)
    assert np.allclose(g["x"].sum(axis=0), seed["x"].sum(axis=0), rtol=1e-9, atol=1e-9)
    sim.close()


def test_backward_restores_the_state_and_stepping_continues():
    sc = adjoint_scene()
    rho0, _, _ = reference(sc)
    seed = seeds(sc, np.random.default_rng(2))
    a = sph.Simulation(sc, precision=sph.SPH_FP32, rho=rho0)
    a.tape(3, DT)
    before, cells_before = a.state(), a.cells()
    a.backward(seed)
    after, cells_after = a.state(), a.cells()
    for k in ("x", "v", "rho", "p", "a", "pw"):
        assert np.array_equal(before[k], after[k]), k
    for k in ("key_f", "order_f", "start_f"):
        assert np.array_equal(cells_before[k], cells_after[k]), k
    a.step(2, DT)
    b = sph.Simulation(sc, precision=sph.SPH_FP32, rho=rho0)
    b.step(5, DT)
    sa, sb = a.state(), b.state()
    for k in ("x", "v", "rho", "pw"):
        assert np.array_equal(sa[k], sb[k]), k
    # a second backward over the same tape gives the same gradients
    a2 = sph.Simulation(sc, precision=sph.SPH_FP32, rho=rho0)
    a2.tape(3, DT)
    g1 = a2.backward(seed)
    g2 = a2.backward(seed)
    for k in ("x", "v", "rho"):
        assert np.array_equal(g1[k], g2[k]), k
    for s_ in (a, b, a2):
        s_.close()


@pytest.mark.parametrize("precision", [sph.SPH_FP32, sph.SPH_FP64_PLAIN])
def test_kept_products_and_the_recompute_give_the_same_gradients(precision):
    """The backward takes each step's products from the tape, or recomputes
    the step when the tape budget left them out: all, none or some kept, the
    state gradients agree bit for bit (the recompute is bit-identical) and
    the parameter gradients to the order of their FP64 atomic sums."""
    sc = adjoint_scene()
    rho0, _, _ = reference(sc)
    seed = seeds(sc, np.random.default_rng(7))
    per_step = sc.n_fluid * 1024 + sc.n_wall * 40 + (8 << 20)  # above one step's products
    grads = []
    for budget in (-1, 0, 2 * per_step):
        sim = sph.Simulation(sc, precision=precision, rho=rho0)
        sim.tape_budget(budget)
        sim.tape(5, DT)
        grads.append(sim.backward(seed))
        sim.close()
    for g in grads[1:]:
        for k in ("x", "v", "rho"):
            assert np.array_equal(g[k], grads[0][k]), k
        for k in ("c0", "gamma_p", "mu"):  # FP64 atomics: summation order varies
            assert g[k] == pytest.approx(grads[0][k], rel=1e-12, abs=1e-300), k
    sim = sph.Simulation(sc, precision=precision, rho=rho0)
    assert lib_status(sph.lib().sph_tape_budget(sim.ctx, -2)) == sph.SPH_ERR_ARG
    sim.close()


def lib_status(st):
    return int(st)


def test_tape_refusals():
    sc = adjoint_scene()
    rho0, _, _ = reference(sc)
    s1 = sph.Simulation(sc, precision=sph.SPH_FP32, rho=rho0)
    st, _ = sph.sph_tape(s1.ctx, 1, DT)
    assert st == sph.SPH_OK
    s1.step(1, DT)  # untaped step
    assert sph.sph_tape(s1.ctx, 1, DT)[0] == sph.SPH_ERR_STATE
    g = sph.sph_adjoint_grad(None, None, None)
    assert sph.sph_backward(s1.ctx, sph.sph_adjoint_seed(None, None, None, None), g) == sph.SPH_ERR_STATE
    s1.close()
    s2 = sph.Simulation(sc, precision=sph.SPH_FP32, rho=rho0)
    assert sph.sph_backward(s2.ctx, sph.sph_adjoint_seed(None, None, None, None), g) == sph.SPH_ERR_STATE
    s2.step(1, DT)
    assert sph.sph_tape(s2.ctx, 1, DT)[0] == sph.SPH_ERR_STATE
    s2.close()
    two = S.two_phase_still_tank()
    s3 = sph.Simulation(two, precision=sph.SPH_FP32)
    assert sph.sph_tape(s3.ctx, 1, DT)[0] == sph.SPH_ERR_UNSUPPORTED
    s3.close()


def test_autograd_function_matches_the_reference(monkeypatch):
    """torch.autograd through SPHRun (device tensors) against the oracle's
    gradient of the same loss.  The device path never converts a tensor to a
    host array (the host marshalling helper raises if it is called)."""
    import torch
    from paper_2110_02621_gb300 import autograd as AG

    def no_host_copy(t):
        raise AssertionError("device tensors went through the host")
    monkeypatch.setattr(AG, "_np", no_host_copy)
    sc = adjoint_scene()
    rho0, normals, sigma0 = reference(sc)
    dev = torch.device("cuda")
    x0 = torch.tensor(sc.fluid_pos, device=dev, requires_grad=True)
    v0 = torch.tensor(sc.fluid_vel, device=dev, requires_grad=True)
    r0 = torch.tensor(rho0, device=dev, requires_grad=True)
    c0 = torch.tensor(sc.c0, dtype=torch.float64, requires_grad=True)
    gp = torch.tensor(sc.gamma_p, dtype=torch.float64, requires_grad=True)
    mu = torch.tensor(sc.phases[0].mu, dtype=torch.float64, requires_grad=True)
    rng = np.random.default_rng(4)
    sx = rng.normal(size=(sc.n_fluid, 3))
    probes = np.arange(0, sc.n_wall, 7)
    xN, vN, rN, pwN = AG.run(x0, v0, r0, c0, gp, mu, sc, 3, DT, precision=sph.SPH_FP64_PLAIN)
    L = (pwN[torch.as_tensor(probes, device=dev)] ** 2).sum() + (xN * torch.tensor(sx, device=dev)).sum()
    L.backward()
    P = A.params_from_scene(sc, normals, sigma0)
    t = lambda a: torch.tensor(np.asarray(a, np.float64))  # noqa: E731
    final = A.run(t(sc.fluid_pos), t(sc.fluid_vel), t(rho0), P, t(sc.c0), t(sc.gamma_p),
                  t(sc.phases[0].mu), 3, DT)
    seed_pw = np.zeros(sc.n_wall)
    seed_pw[probes] = 2.0 * final["pw"].numpy()[probes]
    _, o, _ = A.vjp(sc, normals, sigma0, rho0, 3, DT, {"x": sx, "pw": seed_pw})
    g = {"x": x0.grad.cpu().numpy(), "v": v0.grad.cpu().numpy(), "rho": r0.grad.cpu().numpy(),
         "c0": float(c0.grad), "gamma_p": float(gp.grad), "mu": float(mu.grad)}
    compare(g, o, 1e-8, 1e-8)


def test_adjoint_at_full_size_against_central_differences():
    """The differentiable dam break (188,680 fluid particles, 10 steps, loss =
    sum of squared probe wall pressures), FP64 form: directional derivatives
    along random initial-velocity perturbations of a 2,000-particle subset and
    along c0 and mu, by central differences of the CUDA forward."""
    sc = S.standard("dam_break_adjoint_189k")
    dt = sc.cfl * sc.h / sc.c0
    n = sc.steps
    mask = np.zeros(sc.n_wall)
    mask[sc.probes] = 1.0
    # explicit initial density: the hydrostatic start would make rho^0 depend on c0
    rho0 = oracle.OracleSim(sc).fluid()["rho"].copy()
    sim = sph.Simulation(sc, precision=sph.SPH_FP64_PLAIN, rho=rho0)
    sim.tape(n, dt)
    pw = sim.state()["pw"]
    L0 = float((pw * pw * mask).sum())
    assert L0 > 0
    g = sim.backward({"pw": 2.0 * pw * mask})
    sim.close()

    import copy

    def loss(s):
        q = sph.Simulation(s, precision=sph.SPH_FP64_PLAIN, rho=rho0)
        q.step(n, dt)
        p = q.state()["pw"]
        q.close()
        return float((p * p * mask).sum())

    rng = np.random.default_rng(1)
    sub = rng.choice(sc.n_fluid, 2000, replace=False)
    d = np.zeros((sc.n_fluid, 3))
    d[sub] = rng.normal(size=(2000, 3))
    # the limiter max(U_L - U_R, 0) is only C^1 at U_L = U_R, which a fluid
    # starting at rest sits on: the central difference then errs by O(eps)
    eps = 1e-5
    sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
    sp.fluid_vel = sc.fluid_vel + eps * d
    sm.fluid_vel = sc.fluid_vel - eps * d
    fd = (loss(sp) - loss(sm)) / (2 * eps)
    ad = float((g["v"] * d).sum())
    assert abs(fd - ad) <= 1e-5 * abs(ad), ("v", fd, ad)
    eps = 1e-5 * sc.c0
    sp, sm = copy.deepcopy(sc), copy.deepcopy(sc)
    sp.c0 += eps
    sm.c0 -= eps
    fd = (loss(sp) - loss(sm)) / (2 * eps)
    assert abs(fd - g["c0"]) <= 1e-5 * abs(g["c0"]), ("c0", fd, g["c0"])
    # mu = 0 (inviscid) is the edge of its range: second-order one-sided difference
    assert sc.phases[0].mu == 0.0
    eps = 1e-4
    s1, s2 = copy.deepcopy(sc), copy.deepcopy(sc)
    s1.phases[0].mu = eps
    s2.phases[0].mu = 2 * eps
    fd = (-3.0 * L0 + 4.0 * loss(s1) - loss(s2)) / (2 * eps)
    assert abs(fd - g["mu"]) <= 1e-4 * abs(g["mu"]), ("mu", fd, g["mu"])
