"""torch.autograd.Function over a run of steps of the CUDA library.

``run(x0, v0, rho0, c0, gamma_p, mu, scene, nsteps, dt)`` creates a context
from the given initial state and parameters, tapes ``nsteps`` steps
(sph_tape) and returns the final positions, velocities, densities and wall
pressures as float64 tensors; their backward calls sph_backward, which
recomputes each step from its checkpoint and runs the hand-written adjoint
kernels.  The inputs may live on the CPU or the current CUDA device; the
outputs and gradients live on the device of x0.  On the device the start
state goes to sph_create_device and outputs and gradients come back as
device views: no state passes through the host.  Marshalling only: every step
and every adjoint runs in the CUDA library.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import sph


def _np(t: torch.Tensor) -> np.ndarray:
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy())


class SPHRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, rho0, c0, gamma_p, mu, scene, nsteps, dt, precision):
        phases = [dataclasses.replace(ph, mu=float(mu)) for ph in scene.phases]
        dev = x0.device
        if dev.type == "cuda":
            # device-resident start: sph_create_device copies the tensors on
            # the device (no trip through the host)
            sc = dataclasses.replace(scene, c0=float(c0), gamma_p=float(gamma_p), phases=phases)
            dv = lambda t: t.detach().to(dev, torch.float64).contiguous()  # noqa: E731
            xs, vs, rs = dv(x0), dv(v0), dv(rho0)
            ph = None  # one phase: NULL means phase 0 everywhere
            if len(scene.phases) > 1:
                ph = torch.as_tensor(np.ascontiguousarray(scene.fluid_phase, np.int32)).to(dev)
            sim = sph.Simulation.from_device(sc, xs, vs, rs, ph, precision=precision)
        else:
            sc = dataclasses.replace(scene, fluid_pos=_np(x0), fluid_vel=_np(v0), c0=float(c0),
                                     gamma_p=float(gamma_p), phases=phases)
            sim = sph.Simulation(sc, precision=precision, rho=_np(rho0))
        sim.tape(int(nsteps), float(dt))
        nf, nw = sim.nf, sim.nw
        if dev.type == "cuda":
            outs = [torch.empty((nf, 3), dtype=torch.float64, device=dev),
                    torch.empty((nf, 3), dtype=torch.float64, device=dev),
                    torch.empty(nf, dtype=torch.float64, device=dev),
                    torch.empty(nw, dtype=torch.float64, device=dev)]
            o = sph.sph_state_out(outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(), None,
                                  None, None, None, outs[3].data_ptr(), None, None)
            sph._check(sph.sph_get_state(sim.ctx, o, sph.SPH_DEVICE), sim.ctx)
        else:
            st = sim.state()
            outs = [torch.from_numpy(st[k]) for k in ("x", "v", "rho", "pw")]
        ctx.sim = sim
        ctx.device = dev
        ctx.pdev = (c0.device, gamma_p.device, mu.device)
        return tuple(outs)

    @staticmethod
    def backward(ctx, gx, gv, grho, gpw):
        sim = ctx.sim
        dev = ctx.device
        nf = sim.nf
        if dev.type == "cuda":
            keep = [None if g is None else g.detach().to(dev, torch.float64).contiguous()
                    for g in (gx, gv, grho, gpw)]
            seed = sph.sph_adjoint_seed(*(None if g is None else g.data_ptr() for g in keep))
            out = [torch.empty((nf, 3), dtype=torch.float64, device=dev),
                   torch.empty((nf, 3), dtype=torch.float64, device=dev),
                   torch.empty(nf, dtype=torch.float64, device=dev)]
            grad = sph.sph_adjoint_grad(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
            sph._check(sph.sph_backward(sim.ctx, seed, grad, sph.SPH_DEVICE), sim.ctx)
            params = [float(grad.params[k]) for k in range(3)]
        else:
            seed = {k: None if g is None else _np(g) for k, g in zip(("x", "v", "rho", "pw"),
                                                                     (gx, gv, grho, gpw))}
            g = sim.backward(seed)
            out = [torch.from_numpy(g[k]) for k in ("x", "v", "rho")]
            params = [g["c0"], g["gamma_p"], g["mu"]]
        sim.close()
        ctx.sim = None
        ps = [torch.tensor(p, dtype=torch.float64, device=d) for p, d in zip(params, ctx.pdev)]
        return (out[0], out[1], out[2], ps[0], ps[1], ps[2], None, None, None, None)


def run(x0, v0, rho0, c0, gamma_p, mu, scene, nsteps: int, dt: float, precision: int = sph.SPH_FP32):
    """(x_N, v_N, rho_N, p_w,N) after nsteps taped steps of fixed dt from the
    initial state (x0, v0, rho0) with parameters (c0, gamma_p, mu); scene
    supplies the walls, grid, phase and the remaining constants."""
    as_t = lambda v: v if torch.is_tensor(v) else torch.tensor(float(v), dtype=torch.float64)  # noqa: E731
    return SPHRun.apply(x0, v0, rho0, as_t(c0), as_t(gamma_p), as_t(mu), scene, nsteps, dt, precision)
