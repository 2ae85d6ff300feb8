"""Pins of the FP64 reference adjoint (oracle/adjoint.py), on the CPU.

The PyTorch restatement of the step is checked against the independent C
oracle (same equations, written twice), its autograd gradients against FP64
central differences of the same runs, and both against closed forms: a lone
particle in free fall, and the translation invariance of a wall-free blob."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytest.importorskip("scipy")

import oracle  # noqa: E402
from oracle import adjoint as A  # noqa: E402
from paper_2110_02621_gb300 import scenes as S  # noqa: E402

DT = 1e-4


def adjoint_scene(mu=0.05, reinit_every=2):
    """Small dam break with the fluid pushed 0.3 dp towards the floor and the
    x = 0 wall, jittered by +-0.3 dp, random velocities of 0.3 m/s: every term
    of the step (limiter, viscosity, penalty, reinitialisation) is active."""
    sc = S.dam_break(tank=(0.2, 0.1, 0.12), column=(0.08, 0.1, 0.06), dp=0.01)
    return S.perturbed(sc, jitter=0.3, shift=(-0.3, 0.0, -0.3), vel_scale=0.3, mu=mu,
                       reinit_every=reinit_every)


def c_oracle(sc, rho0=None):
    return oracle.OracleSim(sc, rho=rho0)


def setup(sc):
    ref = c_oracle(sc)
    rho0 = ref.fluid()["rho"].copy()
    normals = ref.wall()["normal"].copy()
    return ref, rho0, normals, ref.sigma0


def test_penalty_is_active_in_the_adjoint_scene():
    sc = adjoint_scene()
    ref, _, normals, _ = setup(sc)
    x = sc.fluid_pos
    xw = sc.wall_pos
    hit = 0
    for i in range(len(x)):
        _, ws = ref.neighbors(i)
        for w in ws:
            rn = np.dot(x[i] - xw[w], normals[w])          # signed delta = 2 rn / dx
            hit += (2 * rn / sc.dp < 1.0) and np.linalg.norm(normals[w]) > 0
    assert hit > 10


def test_torch_penalty_barrier_matches_c_oracle():
    """A particle 0.2 dx behind a fluid-facing wall particle's plane (the C
    oracle's pinned barrier case): the restatement's acceleration, penalty on
    and off, equals the C oracle's."""
    dp = 0.01
    for penalty in (True, False):
        sc = S.Scene(name="pen", dp=dp, h=1.3 * dp, c0=10.0, g=(0, 0, 0), lo=(-0.05, -0.05, -0.05),
                     hi=(0.05, 0.05, 0.05), phases=[S.Phase(eos="linear", penalty=penalty)],
                     fluid_pos=np.array([[0.0, 0.0, -0.2 * dp], [0.0, 0.0, 1.1 * dp]]),
                     fluid_vel=np.zeros((2, 3)), fluid_phase=np.zeros(2, np.int32),
                     wall_pos=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, -dp]]), reinit_every=0)
        rho0 = np.full(2, 1000.5)
        ref = c_oracle(sc, rho0)
        P = A.params_from_scene(sc, ref.wall()["normal"], ref.sigma0)
        t = lambda a: torch.tensor(np.asarray(a, np.float64))  # noqa: E731
        St = A.run(t(sc.fluid_pos), t(sc.fluid_vel), t(rho0), P, t(sc.c0), t(sc.gamma_p),
                   t(sc.phases[0].mu), 0, DT)
        a = ref.fluid()["a"]
        assert np.allclose(St["a"].numpy(), a, rtol=1e-12, atol=1e-12 * np.abs(a).max())


@pytest.mark.parametrize("nsteps", [0, 1, 4])
def test_torch_step_matches_c_oracle(nsteps):
    sc = adjoint_scene()
    ref, rho0, normals, sigma0 = setup(sc)
    P = A.params_from_scene(sc, normals, sigma0)
    t = lambda a: torch.tensor(np.asarray(a, np.float64))  # noqa: E731
    c0, gp, mu = t(sc.c0), t(sc.gamma_p), t(sc.phases[0].mu)
    St = A.run(t(sc.fluid_pos), t(sc.fluid_vel), t(rho0), P, c0, gp, mu, nsteps, DT)
    ref.step(nsteps, DT)
    o, ow = ref.fluid(), ref.wall()

    def rel(a, b):
        return np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300)

    assert rel(St["x"].numpy(), o["x"]) < 1e-13
    assert rel(St["v"].numpy(), o["v"]) < 1e-10
    assert rel(St["rho"].numpy(), o["rho"]) < 1e-12
    assert rel(St["p"].numpy(), o["p"]) < 1e-9
    assert rel(St["a"].numpy(), o["a"]) < 1e-9
    assert rel(St["pw"].numpy(), ow["pw"]) < 1e-9
    # sigma: the C oracle recomputes it at the end of a call
    assert rel(St["sigma"].numpy(), o["sigma"]) < 1e-12


def test_torch_wall_density_floor_matches_c_oracle():
    """Fluid torn to 0.3 rho0 under a roof: the extrapolated p_w of the walls
    above it falls below EOS(rho0/2), where both restatements hold the wall
    density at rho0/2 (and use the inverse EOS elsewhere)."""
    dp = 0.01
    xw = np.array([[i * dp, j * dp, dp] for i in (-1, 0, 1) for j in (-1, 0, 1)])
    sc = S.Scene(name="torn", dp=dp, h=1.3 * dp, c0=10.0, g=(0.0, 0.0, -9.81), lo=(-0.1, -0.1, -0.1),
                 hi=(0.1, 0.1, 0.1), phases=[S.Phase(rho0=1000.0, eos="tait", z_top=0.0)],
                 fluid_pos=np.zeros((1, 3)), fluid_vel=np.zeros((1, 3)),
                 fluid_phase=np.zeros(1, np.int32), wall_pos=xw)
    rho0 = np.array([300.0])
    ref = c_oracle(sc, rho0)
    ow = ref.wall()
    P = A.params_from_scene(sc, ow["normal"], ref.sigma0)
    t = lambda a: torch.tensor(np.asarray(a, np.float64))  # noqa: E731
    St = A.run(t(sc.fluid_pos), t(sc.fluid_vel), t(rho0), P, t(sc.c0), t(sc.gamma_p),
               t(sc.phases[0].mu), 0, DT)
    assert (ow["rhow"][:, 0] == 500.0).any()
    assert np.allclose(St["pw"].numpy(), ow["pw"], rtol=1e-12, atol=0)
    assert np.allclose(St["rhow"].numpy().reshape(len(xw), -1)[:, 0], ow["rhow"][:, 0], rtol=1e-12, atol=0)


def _loss(sc, rho0, normals, sigma0, seed, nsteps, x=None, v=None, r=None, c0=None, gp=None,
          mu=None):
    P = A.params_from_scene(sc, normals, sigma0)
    t = lambda a: torch.tensor(np.asarray(a, np.float64))  # noqa: E731
    S_ = A.run(t(sc.fluid_pos if x is None else x), t(sc.fluid_vel if v is None else v),
               t(rho0 if r is None else r), P, t(sc.c0 if c0 is None else c0),
               t(sc.gamma_p if gp is None else gp), t(sc.phases[0].mu if mu is None else mu),
               nsteps, DT)
    L = 0.0
    for k in ("x", "v", "rho", "pw"):
        if seed.get(k) is not None:
            L += float((S_[k].numpy() * seed[k]).sum())
    return L


def random_seed(sc, rng, probes=None):
    seed = {"x": rng.normal(size=(sc.n_fluid, 3)), "v": rng.normal(size=(sc.n_fluid, 3)),
            "rho": rng.normal(size=sc.n_fluid) * 1e-3, "pw": rng.normal(size=sc.n_wall) * 1e-3}
    return seed


def test_autograd_matches_central_differences():
    sc = adjoint_scene()
    _, rho0, normals, sigma0 = setup(sc)
    rng = np.random.default_rng(7)
    seed = random_seed(sc, rng)
    nsteps = 3
    _, g, _ = A.vjp(sc, normals, sigma0, rho0, nsteps, DT, seed)
    args = dict(sc=sc, rho0=rho0, normals=normals, sigma0=sigma0, seed=seed, nsteps=nsteps)
    checks = []
    # steps balance truncation against the rounding of L (|L| ~ 500); a wall
    # whose fluid support empties makes p_w jump to 0 (no support: p_w = 0),
    # so position steps stay far below the particle spacing
    for name, base, eps in (("x", sc.fluid_pos, 1e-7), ("v", sc.fluid_vel, 1e-5),
                            ("rho", rho0, 1e-2)):
        d = rng.normal(size=np.shape(base))
        key = {"x": "x", "v": "v", "rho": "r"}[name]
        lp = _loss(**args, **{key: base + eps * d})
        lm = _loss(**args, **{key: base - eps * d})
        checks.append((name, (lp - lm) / (2 * eps), float((g[name] * d).sum())))
    for name, key, base, eps in (("c0", "c0", sc.c0, 1e-5 * sc.c0), ("gamma_p", "gp", sc.gamma_p, 1e-3),
                                 ("mu", "mu", sc.phases[0].mu, 1e-4)):
        lp = _loss(**args, **{key: base + eps})
        lm = _loss(**args, **{key: base - eps})
        checks.append((name, (lp - lm) / (2 * eps), float(g[name])))
    for name, fd, ad in checks:
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-8) + 1e-9, (name, fd, ad)
    # every parameter matters in this scene
    assert abs(float(g["gamma_p"])) > 0 and abs(float(g["mu"])) > 0 and abs(float(g["c0"])) > 0


def test_free_fall_closed_form():
    """One particle far from everything: x_N = x0 + v0 T + g T^2/2 exactly under
    KDK with constant g, so dL/dx0 = s_x and dL/dv0 = s_x T + s_v."""
    sc = S.jittered_blob(n=(1, 1, 1), jitter=0.0, vel_scale=0.0)
    sc.g = (0.0, 0.0, -9.81)
    sc.fluid_vel = np.array([[0.1, -0.2, 0.3]])
    rho0 = np.array([1000.0])
    seed = {"x": np.array([[0.3, -1.0, 2.0]]), "v": np.array([[1.5, 0.5, -0.25]])}
    n = 5
    final, g, _ = A.vjp(sc, np.zeros((0, 3)), 1.0, rho0, n, DT, seed)
    T = n * DT
    x_ref = sc.fluid_pos + sc.fluid_vel * T + 0.5 * np.array(sc.g) * T * T
    assert np.allclose(final["x"], x_ref, rtol=0, atol=1e-15)
    assert np.allclose(g["x"], seed["x"], rtol=1e-14)
    assert np.allclose(g["v"], seed["x"] * T + seed["v"], rtol=1e-12)


def test_translation_invariance_of_a_free_blob():
    """Without walls the run commutes with a translation of all particles, so
    the gradients with respect to x0 sum to the seed summed over particles."""
    sc = S.jittered_blob(n=(6, 6, 6), jitter=0.05, vel_scale=0.1)
    sc.phases[0].mu = 0.01
    sc.reinit_every = 2
    ref = c_oracle(sc)
    rho0 = ref.fluid()["rho"]
    rng = np.random.default_rng(3)
    seed = {"x": rng.normal(size=(sc.n_fluid, 3)), "v": rng.normal(size=(sc.n_fluid, 3))}
    _, g, _ = A.vjp(sc, np.zeros((0, 3)), ref.sigma0, rho0, 3, DT, seed)
    assert np.allclose(g["x"].sum(axis=0), seed["x"].sum(axis=0), rtol=1e-9, atol=1e-9)


def periodic_scenes():
    box = S.periodic_box(jitter=0.3, vel_scale=0.3, rho_jitter=0.003, mu=0.05)
    chan = S.perturbed(S.periodic_channel(nz=6), jitter=0.3, shift=(0.0, 0.0, -0.3), vel_scale=0.3, mu=0.05,
                       reinit_every=2)
    return {"box": box, "channel": chan}


@pytest.mark.parametrize("name", ["box", "channel"])
def test_torch_step_matches_c_oracle_with_periodic_axes(name):
    """Nearest images and wrapped drifts: the two restatements agree on a
    periodic box and on a channel periodic along x and y (positions compared
    modulo the period)."""
    sc = periodic_scenes()[name]
    ref, rho0, normals, sigma0 = setup(sc)
    P = A.params_from_scene(sc, normals, sigma0)
    t = lambda a: torch.tensor(np.asarray(a, np.float64))  # noqa: E731
    St = A.run(t(sc.fluid_pos), t(sc.fluid_vel), t(rho0), P, t(sc.c0), t(sc.gamma_p), t(sc.phases[0].mu), 4, DT)
    ref.step(4, DT)
    o, ow = ref.fluid(), ref.wall()
    L = np.array([sc.hi[d] - sc.lo[d] if sc.periodic[d] else np.inf for d in range(3)])
    dx = St["x"].numpy() - o["x"]
    dx = np.where(np.isfinite(L), dx - np.where(np.isfinite(L), L, 0) * np.round(dx / np.where(np.isfinite(L), L, 1)), dx)
    assert np.abs(dx).max() < 1e-13
    assert np.all(St["x"].numpy() >= np.array(sc.lo)) and np.all(St["x"].numpy() < np.array(sc.hi))

    def rel(a, b):
        return np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300)

    assert rel(St["v"].numpy(), o["v"]) < 1e-10
    assert rel(St["rho"].numpy(), o["rho"]) < 1e-12
    assert rel(St["a"].numpy(), o["a"]) < 1e-9
    if sc.n_wall:
        assert rel(St["pw"].numpy(), ow["pw"]) < 1e-9


def test_torch_lone_particle_wraps_like_the_c_oracle():
    """A lone particle crossing the lower x face of a periodic box: both
    restatements wrap its drifted position back into [lo, hi), to the same
    value, (x0 + v t) modulo the period."""
    import dataclasses
    box = S.periodic_box()
    L = np.array(box.hi) - np.array(box.lo)
    x0 = np.array([[0.02 * L[0], 0.5 * L[1], 0.5 * L[2]]])
    v0 = np.array([[-0.5, 0.2, 0.0]])
    sc = dataclasses.replace(box, fluid_pos=x0, fluid_vel=v0, fluid_phase=np.zeros(1, np.int32), rho_init=None,
                             g=(0.0, 0.0, 0.0))
    rho0 = np.array([1000.0])
    ref = c_oracle(sc, rho0)
    P = A.params_from_scene(sc, ref.wall()["normal"], ref.sigma0)
    t = lambda a: torch.tensor(np.asarray(a, np.float64))  # noqa: E731
    dt, n = 1e-3, 20
    St = A.run(t(x0), t(v0), t(rho0), P, t(sc.c0), t(sc.gamma_p), t(sc.phases[0].mu), n, dt)
    ref.step(n, dt)
    xt, xc = St["x"].numpy()[0], ref.fluid()["x"][0]
    assert x0[0, 0] + v0[0, 0] * n * dt < 0.0  # it crossed
    expect = np.array(box.lo) + np.mod(x0[0] + v0[0] * n * dt - np.array(box.lo), L)
    assert np.allclose(xt, expect, rtol=0, atol=1e-13) and np.allclose(xc, expect, rtol=0, atol=1e-13)


def test_periodic_autograd_matches_central_differences():
    sc = periodic_scenes()["box"]
    _, rho0, normals, sigma0 = setup(sc)
    rng = np.random.default_rng(11)
    seed = {"x": rng.normal(size=(sc.n_fluid, 3)), "v": rng.normal(size=(sc.n_fluid, 3)),
            "rho": rng.normal(size=sc.n_fluid) * 1e-3}
    _, g, _ = A.vjp(sc, normals, sigma0, rho0, 3, DT, seed)
    args = dict(sc=sc, rho0=rho0, normals=normals, sigma0=sigma0, seed=seed, nsteps=3)
    for name, key, base, eps in (("x", "x", sc.fluid_pos, 1e-7), ("v", "v", sc.fluid_vel, 1e-5),
                                 ("rho", "r", rho0, 1e-2)):
        d = rng.normal(size=np.shape(base))
        fd = (_loss(**args, **{key: base + eps * d}) - _loss(**args, **{key: base - eps * d})) / (2 * eps)
        ad = float((g[name] * d).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-9, (name, fd, ad)
    lp = _loss(**args, c0=sc.c0 * (1 + 1e-5))
    lm = _loss(**args, c0=sc.c0 * (1 - 1e-5))
    fd = (lp - lm) / (2e-5 * sc.c0)
    assert abs(fd - float(g["c0"])) <= 1e-6 * abs(float(g["c0"])) + 1e-9
