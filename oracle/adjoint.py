"""FP64 reference adjoint of the WCSPH step (arXiv 2110.02621).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/`` this module checks the
CUDA library and is never part of it; only the test suite, the smoke check and
the benchmark's baseline legs may import it.  It shares no code with the CUDA
path (and none with ``sph_oracle.c`` either: it is a second, independent
restatement of the same step).

What it computes: the kick-drift-kick step of Sec. 2.6 with the Riemann
continuity and momentum equations (Eqs. (LRstates), (RSsolution),
(SPH_star_massConservation), (SPH_star_momentumConservation)), the wall
pressure of Eq. (wallPressure), the wall Riemann pressure of Eq. (RSatWall),
the penalty force of Eqs. (SPH_penaltyMethodTerm), (symbc) and
(deltaForPenalty), the density reinitialisation of Eq. (eqrhosum) and the
Morris viscosity, in the same order and with the same readings as the C
oracle, written with plain PyTorch CPU tensor operations in float64 so that
``torch.autograd`` differentiates it.  Sums over neighbours are written as
sums over explicit pair lists (index_add), the lists found by a k-d tree on the
positions of the step (pairs with 0 < r < 2h).  The adjoint (vector-Jacobian
product) of a whole run is then ``torch.autograd.grad`` of a scalar loss.

Scope: one phase, continuity density, fixed walls, a fixed time step (the
adjoint treats dt as a constant of the run).  The state of a run is
(x, v, rho, a, p_w, sigma): a, p_w and sigma are carried from one step to the
next exactly as in the C oracle (a^n for the first half kick, the previous
wall pressure for the continuity equation, sigma(r^n) for the
reinitialisation), and ``create`` computes them from (x^0, v^0, rho^0).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np
import torch
from scipy.spatial import cKDTree

F64 = torch.float64


@dataclasses.dataclass
class Params:
    """Constants of a run.  c0, gamma_p and mu may be tensors (requires_grad)."""
    dp: float
    h: float
    rho0: float
    tait: bool
    gamma_tait: float
    g: torch.Tensor          # (3,)
    penalty: bool
    reinit_every: int
    sigma0: float            # lattice number density (reading of Sec. 2.5)
    normals: torch.Tensor    # (nw, 3) wall normals, Eq. (normalVectors)
    xw: torch.Tensor         # (nw, 3) wall positions
    lo: Optional[torch.Tensor] = None      # (3,) grid origin
    period: Optional[torch.Tensor] = None  # (3,) period of each periodic axis, 0 elsewhere


def params_from_scene(sc, normals: np.ndarray, sigma0: float) -> Params:
    assert len(sc.phases) == 1 and sc.phases[0].density == "continuity"
    ph = sc.phases[0]
    return Params(dp=sc.dp, h=sc.h, rho0=ph.rho0, tait=ph.eos == "tait",
                  gamma_tait=sc.gamma_tait, g=torch.tensor(sc.g, dtype=F64),
                  penalty=bool(ph.penalty), reinit_every=sc.reinit_every,
                  sigma0=sigma0, normals=torch.tensor(normals, dtype=F64),
                  xw=torch.tensor(np.asarray(sc.wall_pos, np.float64).reshape(-1, 3)),
                  lo=torch.tensor(sc.lo, dtype=F64),
                  period=torch.tensor([(sc.hi[d] - sc.lo[d]) if getattr(sc, "periodic", (0, 0, 0))[d] else 0.0
                                       for d in range(3)], dtype=F64))


# ------------------------------------------------------------ periodic axes
def _periodic(P) -> bool:
    return P is not None and P.period is not None and bool((P.period > 0).any())


def image(r, P):
    """The nearest periodic image of pair vectors r (n, 3): a shift by whole
    periods, constant in the positions (derivative 1)."""
    if not _periodic(P):
        return r
    L = torch.where(P.period > 0, P.period, torch.ones_like(P.period))
    k = torch.where(P.period > 0, torch.round(r.detach() / L), torch.zeros_like(r))
    return r - k * L


def wrap(x, P):
    """Positions wrapped into [lo, lo + period) along the periodic axes."""
    if not _periodic(P):
        return x
    L = torch.where(P.period > 0, P.period, torch.ones_like(P.period))
    k = torch.where(P.period > 0, torch.floor((x.detach() - P.lo) / L), torch.zeros_like(x))
    return x - k * L


# ------------------------------------------------------------ kernel, EOS
def W(r, h):
    """3-D Wendland C2, support 2h: 21/(16 pi h^3) (1 - q/2)^4 (2q + 1)."""
    q = r / h
    t = torch.clamp(1.0 - 0.5 * q, min=0.0)
    return 21.0 / (16.0 * math.pi * h ** 3) * t ** 4 * (2.0 * q + 1.0)


def dWdr(r, h):
    """dW/dr = -5 alpha q (1 - q/2)^3 / h."""
    q = r / h
    t = torch.clamp(1.0 - 0.5 * q, min=0.0)
    return -5.0 * 21.0 / (16.0 * math.pi * h ** 3) * q * t ** 3 / h


def eos_p(rho, P: Params, c0):
    """Eq. (EoS) (linear) or Tait."""
    if P.tait:
        return P.rho0 * c0 ** 2 / P.gamma_tait * ((rho / P.rho0) ** P.gamma_tait - 1.0)
    return c0 ** 2 * (rho - P.rho0)


def eos_rho(p, P: Params, c0):
    if P.tait:
        return P.rho0 * (1.0 + P.gamma_tait * p / (P.rho0 * c0 ** 2)) ** (1.0 / P.gamma_tait)
    return P.rho0 + p / c0 ** 2


def riemann(rhoL, UL, pL, rhoR, UR, pR, c):
    """Eqs. (LRstates), (RSsolution) with the limiter beta = min(3 max(UL - UR, 0), c).
    Returns (U*, p*, U_bar)."""
    rs = rhoL + rhoR
    rho_bar = 0.5 * rs
    U_bar = (rhoL * UL + rhoR * UR) / rs
    P_bar = (rhoL * pR + rhoR * pL) / rs
    Ustar = U_bar + 0.5 * (pL - pR) / (c * rho_bar)
    beta = torch.minimum(3.0 * torch.clamp(UL - UR, min=0.0), c * torch.ones_like(UL))
    pstar = P_bar + rhoL * rhoR * beta * (UL - UR) / rs
    return Ustar, pstar, U_bar


# ------------------------------------------------------------ pair lists
def _torus(pts: np.ndarray, P):
    """Points shifted into the box [0, size) of a k-d tree that is toroidal
    along the periodic axes (the others get a box far larger than the
    points' extent, so that nothing wraps there), and the box."""
    lo, per = P.lo.numpy(), P.period.numpy()
    if len(pts) == 0:
        return pts, np.where(per > 0, per, 1.0)
    base = pts.min(axis=0)
    box = np.where(per > 0, per, 4.0 * (np.ptp(pts, axis=0) + 1.0))
    shifted = np.where(per > 0, np.mod(pts - lo, np.where(per > 0, per, 1.0)), pts - base)
    return np.minimum(shifted, np.nextafter(box, 0)), box


def fluid_pairs(x: torch.Tensor, h: float, P=None):
    """Directed pairs (i, j), i != j, with 0 < |x_i - x_j| < 2h (nearest
    images along periodic axes)."""
    xn = x.detach().numpy()
    if _periodic(P):
        sh, box = _torus(xn, P)
        tree = cKDTree(sh, boxsize=box)
    else:
        tree = cKDTree(xn)
    pr = tree.query_pairs(2.0 * h, output_type="ndarray")
    if len(pr) == 0:
        z = torch.zeros(0, dtype=torch.int64)
        return z, z
    d = image(torch.from_numpy(xn[pr[:, 0]] - xn[pr[:, 1]]), P).numpy()
    r2 = (d * d).sum(axis=1)
    pr = pr[(r2 < 4.0 * h * h) & (r2 > 0.0)]
    i = np.concatenate([pr[:, 0], pr[:, 1]])
    j = np.concatenate([pr[:, 1], pr[:, 0]])
    return torch.from_numpy(i), torch.from_numpy(j)


def wall_pairs(x: torch.Tensor, xw: torch.Tensor, h: float, P=None):
    """Pairs (fluid i, wall w) with 0 < |x_i - x_w| < 2h (nearest images
    along periodic axes)."""
    if xw.shape[0] == 0 or x.shape[0] == 0:
        z = torch.zeros(0, dtype=torch.int64)
        return z, z
    xn, wn = x.detach().numpy(), xw.numpy()
    if _periodic(P):
        sh, box = _torus(np.concatenate([wn, xn]), P)
        lists = cKDTree(sh[: len(wn)], boxsize=box).query_ball_point(sh[len(wn):], 2.0 * h)
    else:
        lists = cKDTree(wn).query_ball_point(xn, 2.0 * h)
    i = np.repeat(np.arange(len(lists)), [len(l) for l in lists])
    w = np.concatenate([np.asarray(l, np.int64) for l in lists]) if len(i) else np.zeros(0, np.int64)
    d = image(torch.from_numpy(xn[i] - wn[w]), P).numpy()
    r2 = (d * d).sum(axis=1)
    keep = (r2 < 4.0 * h * h) & (r2 > 0.0)
    return torch.from_numpy(i[keep]), torch.from_numpy(w[keep])


def _geom(xa, xb, ia, ib, P=None):
    rij = image(xa[ia] - xb[ib], P)
    r = torch.sqrt((rij * rij).sum(dim=1))
    return rij, r


# ------------------------------------------------------------ operators
def continuity(x, v, rho, p, pw, rhow, P: Params, c0, pairs):
    """d rho_i/dt, Eq. (SPH_star_massConservation):
    2 rho_i sum_j (m_j/rho_j) (v_i - v*).grad_i W_ij, with v* from the Riemann
    solution along e_ij = -r_ij/r; walls with v_w = 0, (rho_w, p_w)."""
    (fi, fj), (wi, ww) = pairs
    m = P.rho0 * P.dp ** 3
    out = torch.zeros_like(rho)

    def add(i, rij, r, rho_j, p_j, v_j):
        e = -rij / r[:, None]
        gw = (dWdr(r, P.h) / r)[:, None] * rij
        v_i = v[i]
        UL = (v_i * e).sum(dim=1)
        UR = (v_j * e).sum(dim=1)
        Ustar, _, U_bar = riemann(rho[i], UL, p[i], rho_j, UR, p_j, c0)
        vmix = (rho[i][:, None] * v_i + rho_j[:, None] * v_j) / (rho[i] + rho_j)[:, None]
        vstar = Ustar[:, None] * e + (vmix - U_bar[:, None] * e)
        dot = ((v_i - vstar) * gw).sum(dim=1)
        out.index_add_(0, i, 2.0 * rho[i] * (m / rho_j) * dot)

    rij, r = _geom(x, x, fi, fj, P)
    add(fi, rij, r, rho[fj], p[fj], v[fj])
    rij, r = _geom(x, P.xw, wi, ww, P)
    add(wi, rij, r, rhow[ww], pw[ww], torch.zeros_like(rij))
    return out


def wall_pressure(x, rho, p, P: Params, c0, wpairs, nw):
    """Eq. (wallPressure), fixed walls, rho_f weighting the g term:
    p_w = sum_f (p_f + rho_f g.r_wf) W_wf / sum_f W_wf, r_wf = r_w - r_f;
    no support: p_w = 0.  rho_w = EOS^-1(p_w), at least rho0/2."""
    wi, ww = wpairs
    rwf = image(P.xw[ww] - x[wi], P)
    r = torch.sqrt((rwf * rwf).sum(dim=1))
    Wk = W(r, P.h)
    num = torch.zeros(nw, dtype=F64).index_add(0, ww, (p[wi] + rho[wi] * (rwf @ P.g)) * Wk)
    den = torch.zeros(nw, dtype=F64).index_add(0, ww, Wk)
    has = den > 0.0
    pw = torch.where(has, num / torch.where(has, den, torch.ones_like(den)), torch.zeros_like(den))
    # rho_w kept at or above rho0/2: EOS^-1 of max(p_w, EOS(rho0/2))
    p_half = eos_p(0.5 * P.rho0 * torch.ones_like(pw), P, c0)
    return pw, eos_rho(torch.maximum(pw, p_half), P, c0)


def momentum(x, v, rho, p, pw, rhow, P: Params, c0, gamma_p, mu, pairs):
    """Eq. (SPH_star_momentumConservation): -2 sum_j m_j p*/(rho_i rho_j) grad_i W_ij
    (fluid p* from Eq. (RSsolution) with the limiter, wall p* from Eq. (RSatWall)),
    the penalty force F_p (delta = 2 r_iw.n_w/dx signed, lambda =
    (1-delta)^2/dx for delta < 1, P = gamma_p lambda |p_i e_iw.n_w|, times
    dx^3 |r|^-2 dW/dr) through the fluid-facing wall particles (some fluid of
    their support on the side the normal points to), the Morris viscosity
    with mu_i + mu_j, and g."""
    (fi, fj), (wi, ww) = pairs
    m = P.rho0 * P.dp ** 3
    eta2 = 0.01 * P.h ** 2
    a = torch.zeros_like(x)
    # fluid-fluid
    rij, r = _geom(x, x, fi, fj, P)
    e = -rij / r[:, None]
    F = dWdr(r, P.h) / r
    gw = F[:, None] * rij
    UL = (v[fi] * e).sum(dim=1)
    UR = (v[fj] * e).sum(dim=1)
    _, pstar, _ = riemann(rho[fi], UL, p[fi], rho[fj], UR, p[fj], c0)
    a = a.index_add(0, fi, (-2.0 * m * pstar / (rho[fi] * rho[fj]))[:, None] * gw)
    kv = m * (2.0 * mu) * (rij * gw).sum(dim=1) / (rho[fi] * rho[fj] * (r * r + eta2))
    a = a.index_add(0, fi, kv[:, None] * (v[fi] - v[fj]))
    # fluid-wall
    rij, r = _geom(x, P.xw, wi, ww, P)
    F = dWdr(r, P.h) / r
    gw = F[:, None] * rij
    rho_i, p_i, rho_w, p_w = rho[wi], p[wi], rhow[ww], pw[ww]
    pstar = (rho_i * p_w + rho_w * p_i) / (rho_i + rho_w)
    a = a.index_add(0, wi, (-2.0 * m * pstar / (rho_i * rho_w))[:, None] * gw)
    kv = m * (2.0 * mu) * (rij * gw).sum(dim=1) / (rho_i * rho_w * (r * r + eta2))
    a = a.index_add(0, wi, kv[:, None] * v[wi])
    if P.penalty:
        nw_ = P.normals[ww]
        rn = (rij * nw_).sum(dim=1)                      # r_iw . n_w
        facing = torch.zeros(P.normals.shape[0], dtype=F64).index_add(0, ww, (rn > 0.0).to(F64)) > 0.0
        e = -rij / r[:, None]
        en = (e * nw_).sum(dim=1)
        dx = P.dp
        delta = 2.0 * rn / dx
        act = facing[ww] & (delta < 1.0) & (r > 1e-6 * dx)
        lam = torch.where(act, (1.0 - delta) ** 2 / dx, torch.zeros_like(delta))
        Ppen = gamma_p * lam * torch.abs(p_i * en)
        k = -2.0 * m / (rho_i * rho_w) * Ppen * dx ** 3 / (r * r) * dWdr(r, P.h)
        a = a.index_add(0, wi, k[:, None] * nw_)
    return a + P.g


def number_density(x, P: Params, pairs, n):
    """sigma_i = W(0) + sum_j W_ij + sum_w W_iw (one phase: all fluid)."""
    (fi, fj), (wi, ww) = pairs
    s = torch.full((n,), float(W(torch.tensor(0.0, dtype=F64), P.h)), dtype=F64)
    _, r = _geom(x, x, fi, fj, P)
    s = s.index_add(0, fi, W(r, P.h))
    _, r = _geom(x, P.xw, wi, ww, P)
    return s.index_add(0, wi, W(r, P.h))


def reinit(rho, sigma, P: Params):
    """Eq. (eqrhosum): rho = rho_num + max(0, rho* - rho_num) rho0/rho*,
    rho_num = rho0 sigma/sigma0."""
    rho_num = P.rho0 * sigma / P.sigma0
    return rho_num + torch.clamp(rho - rho_num, min=0.0) * P.rho0 / rho


# ------------------------------------------------------------ runs
def create(x, v, rho, P: Params, c0, gamma_p, mu) -> Dict[str, torch.Tensor]:
    """The state after sph_create: p^0 = EOS(rho^0), the wall pressure, a^0
    and sigma(r^0) of the initial positions."""
    nw = P.xw.shape[0]
    x = wrap(x, P)
    pairs = (fluid_pairs(x, P.h, P), wall_pairs(x, P.xw, P.h, P))
    p = eos_p(rho, P, c0)
    pw, rhow = wall_pressure(x, rho, p, P, c0, pairs[1], nw)
    a = momentum(x, v, rho, p, pw, rhow, P, c0, gamma_p, mu, pairs)
    sigma = number_density(x, P, pairs, x.shape[0])
    return {"x": x, "v": v, "rho": rho, "p": p, "a": a, "pw": pw, "rhow": rhow, "sigma": sigma}


def step(S, P: Params, c0, gamma_p, mu, dt: float, do_reinit: bool):
    """One kick-drift-kick step (Sec. 2.6), in the order of the C oracle."""
    nw = P.xw.shape[0]
    rho, p = S["rho"], S["p"]
    if do_reinit:
        rho = reinit(rho, S["sigma"], P)
        p = eos_p(rho, P, c0)
    vh = S["v"] + 0.5 * dt * S["a"]
    x = wrap(S["x"] + dt * vh, P)
    pairs = (fluid_pairs(x, P.h, P), wall_pairs(x, P.xw, P.h, P))
    drdt = continuity(x, vh, rho, p, S["pw"], S["rhow"], P, c0, pairs)
    rho1 = rho + dt * drdt
    p1 = eos_p(rho1, P, c0)
    pw, rhow = wall_pressure(x, rho1, p1, P, c0, pairs[1], nw)
    a = momentum(x, vh, rho1, p1, pw, rhow, P, c0, gamma_p, mu, pairs)
    v1 = vh + 0.5 * dt * a
    sigma = number_density(x, P, pairs, x.shape[0])
    return {"x": x, "v": v1, "rho": rho1, "p": p1, "a": a, "pw": pw, "rhow": rhow,
            "sigma": sigma, "drho_dt": drdt}


def run(x0, v0, rho0, P: Params, c0, gamma_p, mu, nsteps: int, dt: float,
        first_step: int = 0):
    S = create(x0, v0, rho0, P, c0, gamma_p, mu)
    for k in range(nsteps):
        n = first_step + k
        S = step(S, P, c0, gamma_p, mu, dt, P.reinit_every > 0 and n % P.reinit_every == 0)
    return S


def vjp(sc, normals, sigma0, rho0: np.ndarray, nsteps: int, dt: float,
        seed: Dict[str, np.ndarray], c0: Optional[float] = None,
        gamma_p: Optional[float] = None, mu: Optional[float] = None):
    """Gradient of L = sum(seed_x . x_N) + sum(seed_v . v_N) + sum(seed_rho rho_N)
    + sum(seed_pw p_w,N) with respect to (x^0, v^0, rho^0, c0, gamma_p, mu).
    Returns (final state as numpy, gradients as numpy / floats)."""
    P = params_from_scene(sc, normals, sigma0)
    x0 = torch.tensor(np.asarray(sc.fluid_pos, np.float64), requires_grad=True)
    v0 = torch.tensor(np.asarray(sc.fluid_vel, np.float64), requires_grad=True)
    r0 = torch.tensor(np.asarray(rho0, np.float64), requires_grad=True)
    tc0 = torch.tensor(sc.c0 if c0 is None else c0, dtype=F64, requires_grad=True)
    tgp = torch.tensor(sc.gamma_p if gamma_p is None else gamma_p, dtype=F64, requires_grad=True)
    tmu = torch.tensor(sc.phases[0].mu if mu is None else mu, dtype=F64, requires_grad=True)
    S = run(x0, v0, r0, P, tc0, tgp, tmu, nsteps, dt)
    L = torch.zeros((), dtype=F64)
    for k, t in (("x", S["x"]), ("v", S["v"]), ("rho", S["rho"]), ("pw", S["pw"])):
        if seed.get(k) is not None:
            L = L + (torch.tensor(np.asarray(seed[k], np.float64)) * t).sum()
    grads = torch.autograd.grad(L, [x0, v0, r0, tc0, tgp, tmu], allow_unused=True)
    out = {}
    for name, g in zip(("x", "v", "rho", "c0", "gamma_p", "mu"), grads):
        out[name] = (np.zeros(()) if g is None else g.detach().numpy())
    final = {k: t.detach().numpy() for k, t in S.items()}
    return final, out, float(L.detach())
