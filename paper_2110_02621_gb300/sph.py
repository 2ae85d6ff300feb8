"""ctypes binding of libsph_gb300.so (include/sph.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no CPU fallback.  ``Simulation`` wraps a context for one scene.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

SPH_OK, SPH_ERR_ARG, SPH_ERR_CUDA, SPH_ERR_OOM = 0, 1, 2, 3
SPH_ERR_DOMAIN, SPH_ERR_NONFINITE, SPH_ERR_STATE, SPH_ERR_UNSUPPORTED = 4, 5, 6, 7
SPH_FP32, SPH_FP64_PLAIN = 0, 1
SPH_HOST, SPH_DEVICE = 0, 1
STATUS_NAMES = {0: "SPH_OK", 1: "SPH_ERR_ARG", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_OOM",
                4: "SPH_ERR_DOMAIN", 5: "SPH_ERR_NONFINITE", 6: "SPH_ERR_STATE",
                7: "SPH_ERR_UNSUPPORTED", 8: "SPH_ERR_CAPACITY"}
_EOS = {"linear": 0, "tait": 1}
_DENSITY = {"continuity": 0, "summation": 1}
_REINIT = {"none": 0, "free_surface": 1, "internal": 2}
EXPORTS = ("sph_create", "sph_step", "sph_reinit_density", "sph_get_state",
           "sph_grid_info", "sph_get_cells", "sph_diagnostics", "sph_counters",
           "sph_last_error", "sph_destroy", "sph_bin_sort", "sph_bin_sort_noalloc",
           "sph_profile", "sph_profile_read", "sph_tape", "sph_backward", "sph_step_async",
           "sph_sync", "sph_diagnostics_async", "sph_set_excitation", "sph_time",
           "sph_probe_pressure", "sph_gauge_height", "sph_tape_budget", "sph_get_neighbors",
           "sph_create_device")
SPH_GAUGE_MAX_SAMPLES = 65536
SPH_GAUGE_MAX_LINES = 65535
SPH_ERR_CAPACITY = 8
SPH_BIN_SORT_NOALLOC_SCRATCH = 32 << 20
KERNEL_KINDS = ("begin_step", "predict", "scan", "scatter", "gather", "neighbors",
                "continuity", "wall_pressure", "momentum", "other", "adj_momentum",
                "adj_continuity", "adj_wall", "adj_other")
SPH_NK = len(KERNEL_KINDS)


class sph_phase(C.Structure):
    _fields_ = [("rho0", C.c_double), ("mu", C.c_double), ("z_top", C.c_double),
                ("eos", C.c_int32), ("density", C.c_int32), ("reinit", C.c_int32),
                ("penalty", C.c_int32)]


class sph_params(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("c0", C.c_double),
                ("gamma_tait", C.c_double), ("gamma_p", C.c_double), ("cfl", C.c_double),
                ("g", C.c_double * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("n_phases", C.c_int32), ("reinit_every", C.c_int32),
                ("phase", sph_phase * 2), ("precision", C.c_int32), ("dim", C.c_int32),
                ("periodic", C.c_int32)]


class sph_fluid(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("vel", C.c_void_p),
                ("rho", C.c_void_p), ("phase", C.c_void_p)]


class sph_wall(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p)]


class sph_state_out(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("pos", "vel", "rho", "p", "acc", "drho_dt",
                                          "sigma", "pw", "rhow", "normal")]


class sph_adjoint_seed(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("x", "v", "rho", "pw")]


class sph_adjoint_grad(C.Structure):
    _fields_ = [("x", C.c_void_p), ("v", C.c_void_p), ("rho", C.c_void_p),
                ("params", C.c_double * 3)]


class SphError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


_lib_path = None


def use_library(path: Optional[str]) -> Optional[str]:
    """Bind to another build of the library from now on (e.g. the
    index-checking build, build.build(check=True)); None = the default.
    Returns the previous choice.  Contexts of the previous library must be
    destroyed first."""
    global _lib, _lib_path
    prev = _lib_path
    _lib, _lib_path = None, path
    return prev


def lib() -> C.CDLL:
    """Load libsph_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _lib_path or _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -m paper_2110_02621_gb300.build` (nvcc, sm_103a)")
        L = C.CDLL(path)
        p, i32, i64, d, st = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int
        L.sph_create.argtypes = [p, p, p, p, C.POINTER(p)]
        L.sph_create_device.argtypes = [p, p, p, p, C.POINTER(p)]
        L.sph_step.argtypes = [p, i32, d, p]
        L.sph_reinit_density.argtypes = [p]
        L.sph_get_state.argtypes = [p, p, i32]
        L.sph_grid_info.argtypes = [p, p, p, p]
        L.sph_get_cells.argtypes = [p] * 7
        L.sph_diagnostics.argtypes = [p, p]
        L.sph_counters.argtypes = [p, p, p]
        L.sph_last_error.argtypes = [p]
        L.sph_last_error.restype = C.c_char_p
        L.sph_destroy.argtypes = [p]
        L.sph_destroy.restype = None
        L.sph_bin_sort.argtypes = [p, i64, p, d, p, p, p, p, p]
        L.sph_bin_sort_noalloc.argtypes = [p, i64, p, d, p, p, p, p, p]
        L.sph_profile.argtypes = [p, C.c_uint32]
        L.sph_profile_read.argtypes = [p, p, p, p]
        L.sph_tape.argtypes = [p, i32, d, p]
        L.sph_step_async.argtypes = [p, i32, d]
        L.sph_sync.argtypes = [p, p]
        L.sph_diagnostics_async.argtypes = [p, p, i32]
        L.sph_set_excitation.argtypes = [p, p, d]
        L.sph_time.argtypes = [p, p]
        L.sph_backward.argtypes = [p, p, p, i32]
        L.sph_probe_pressure.argtypes = [p, p, i32, p, p, i32]
        L.sph_tape_budget.argtypes = [p, i64]
        L.sph_gauge_height.argtypes = [p, p, i32, d, p, i32]
        L.sph_get_neighbors.argtypes = [p, p, p, i64, p, p, i64, p]
        for name in EXPORTS:
            if name not in ("sph_last_error", "sph_destroy"):
                getattr(L, name).restype = st
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _check(status: int, ctx=None):
    if status != SPH_OK:
        msg = lib().sph_last_error(ctx)
        raise SphError(status, msg.decode() if msg else "")


def make_params(scene, precision: int = SPH_FP32) -> sph_params:
    P = sph_params()
    P.dp, P.h, P.c0 = scene.dp, scene.h, scene.c0
    P.gamma_tait, P.gamma_p, P.cfl = scene.gamma_tait, scene.gamma_p, scene.cfl
    for d in range(3):
        P.g[d], P.lo[d], P.hi[d] = scene.g[d], scene.lo[d], scene.hi[d]
    P.n_phases = len(scene.phases)
    P.reinit_every = scene.reinit_every
    for k, ph in enumerate(scene.phases):
        P.phase[k] = sph_phase(rho0=ph.rho0, mu=ph.mu, z_top=ph.z_top, eos=_EOS[ph.eos],
                               density=_DENSITY[ph.density], reinit=_REINIT[ph.reinit],
                               penalty=int(bool(ph.penalty)))
    P.precision = precision
    P.dim = getattr(scene, "dim", 3)
    per = getattr(scene, "periodic", (0, 0, 0))
    P.periodic = sum(1 << d for d in range(3) if per[d])
    return P


def current_stream_handle() -> int:
    """The raw cudaStream_t of torch's current stream (0 without torch/CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


# ------------------------------------------------------------ raw C calls
def sph_create(params: sph_params, fluid: sph_fluid, wall: Optional[sph_wall],
               stream: int = 0):
    ctx = C.c_void_p()
    st = lib().sph_create(C.byref(params), C.byref(fluid),
                          C.byref(wall) if wall is not None else None,
                          C.c_void_p(stream), C.byref(ctx))
    return st, ctx


def sph_create_device(params: sph_params, fluid: sph_fluid, wall: Optional[sph_wall],
                      stream: int = 0):
    """sph_create with fluid arrays that are device memory."""
    ctx = C.c_void_p()
    st = lib().sph_create_device(C.byref(params), C.byref(fluid),
                                 C.byref(wall) if wall is not None else None,
                                 C.c_void_p(stream), C.byref(ctx))
    return st, ctx


def sph_step(ctx, nsteps: int, dt: float = 0.0):
    out = C.c_double()
    st = lib().sph_step(ctx, int(nsteps), float(dt), C.byref(out))
    return st, out.value


def sph_reinit_density(ctx):
    return lib().sph_reinit_density(ctx)


def sph_get_state(ctx, out: sph_state_out, where: int = SPH_HOST):
    return lib().sph_get_state(ctx, C.byref(out), int(where))


def sph_grid_info(ctx):
    dims = np.zeros(3, np.int32)
    nc = C.c_int64()
    cs = C.c_double()
    st = lib().sph_grid_info(ctx, _ptr(dims), C.byref(nc), C.byref(cs))
    return st, dims, nc.value, cs.value


def sph_get_cells(ctx, *arrays):
    return lib().sph_get_cells(ctx, *(_ptr(a) for a in arrays))


def sph_get_neighbors(ctx, f_off, f_ids, f_cap: int, w_off, w_ids, w_cap: int, overflow):
    return lib().sph_get_neighbors(ctx, _ptr(f_off), _ptr(f_ids), int(f_cap), _ptr(w_off), _ptr(w_ids),
                                   int(w_cap), _ptr(overflow))


def sph_diagnostics(ctx, out: np.ndarray):
    return lib().sph_diagnostics(ctx, _ptr(out))


def sph_counters(ctx):
    steps, active = C.c_int64(), C.c_int64()
    st = lib().sph_counters(ctx, C.byref(steps), C.byref(active))
    return st, steps.value, active.value


def sph_last_error(ctx=None) -> str:
    msg = lib().sph_last_error(ctx)
    return msg.decode() if msg else ""


def sph_destroy(ctx):
    lib().sph_destroy(ctx)


def sph_bin_sort(pos_dev: int, n: int, lo, h: float, dims, key_dev: int, order_dev: int,
                 start_dev: int, stream: int = 0):
    lo_a = (C.c_double * 3)(*lo)
    dims_a = (C.c_int32 * 3)(*[int(v) for v in dims])
    return lib().sph_bin_sort(C.c_void_p(pos_dev), int(n), lo_a, float(h), dims_a,
                              C.c_void_p(key_dev), C.c_void_p(order_dev),
                              C.c_void_p(start_dev), C.c_void_p(stream))


def sph_bin_sort_noalloc(pos_dev: int, n: int, lo, h: float, dims, key_dev: int, order_dev: int,
                         start_dev: int, stream: int = 0):
    lo_a = (C.c_double * 3)(*lo)
    dims_a = (C.c_int32 * 3)(*[int(v) for v in dims])
    return lib().sph_bin_sort_noalloc(C.c_void_p(pos_dev), int(n), lo_a, float(h), dims_a,
                                      C.c_void_p(key_dev), C.c_void_p(order_dev),
                                      C.c_void_p(start_dev), C.c_void_p(stream))


def sph_profile(ctx, kind_mask: int):
    return lib().sph_profile(ctx, int(kind_mask))


def sph_profile_read(ctx):
    ms = np.zeros(SPH_NK)
    timed = np.zeros(SPH_NK, np.int64)
    launches = np.zeros(SPH_NK, np.int64)
    st = lib().sph_profile_read(ctx, _ptr(ms), _ptr(timed), _ptr(launches))
    return st, ms, timed, launches


def sph_step_async(ctx, nsteps: int, dt: float = 0.0):
    return lib().sph_step_async(ctx, int(nsteps), float(dt))


def sph_sync(ctx):
    last = C.c_double(0.0)
    st = lib().sph_sync(ctx, C.byref(last))
    return st, last.value


def sph_diagnostics_async(ctx, out_ptr: int, where: int = SPH_HOST):
    return lib().sph_diagnostics_async(ctx, out_ptr, int(where))


def sph_probe_pressure(ctx, pts_ptr, n: int, p_ptr, w_ptr, where: int = SPH_HOST):
    return lib().sph_probe_pressure(ctx, pts_ptr, int(n), p_ptr, w_ptr, int(where))


def sph_gauge_height(ctx, gauges_ptr, n: int, dz: float, H_ptr, where: int = SPH_HOST):
    return lib().sph_gauge_height(ctx, gauges_ptr, int(n), float(dz), H_ptr, int(where))


def sph_tape(ctx, nsteps: int, dt: float = 0.0):
    last = C.c_double(0.0)
    st = lib().sph_tape(ctx, int(nsteps), float(dt), C.byref(last))
    return st, last.value


def sph_backward(ctx, seed: sph_adjoint_seed, grad: sph_adjoint_grad, where: int = SPH_HOST):
    return lib().sph_backward(ctx, C.byref(seed), C.byref(grad), int(where))


# ------------------------------------------------------------ convenience
class Simulation:
    """One simulation context on the current CUDA device and stream."""

    def __init__(self, scene, precision: int = SPH_FP32, rho: Optional[np.ndarray] = None,
                 stream: Optional[int] = None):
        self.scene = scene
        self.precision = precision
        self.nf, self.nw = scene.n_fluid, scene.n_wall
        self._x = np.ascontiguousarray(scene.fluid_pos, np.float64)
        self._v = np.ascontiguousarray(scene.fluid_vel, np.float64)
        self._ph = np.ascontiguousarray(scene.fluid_phase, np.int32)
        self._xw = np.ascontiguousarray(scene.wall_pos, np.float64).reshape(-1, 3)
        if rho is None:
            rho = getattr(scene, "rho_init", None)
        self._rho = None if rho is None else np.ascontiguousarray(rho, np.float64)
        self.params = make_params(scene, precision)
        fluid = sph_fluid(self.nf, _ptr(self._x), _ptr(self._v), _ptr(self._rho), _ptr(self._ph))
        wall = sph_wall(self.nw, _ptr(self._xw))
        self.stream = current_stream_handle() if stream is None else stream
        st, ctx = sph_create(self.params, fluid, wall, self.stream)
        _check(st, None)
        self.ctx = ctx

    @classmethod
    def from_device(cls, scene, x, v=None, rho=None, phase=None, precision: int = SPH_FP32,
                    stream: Optional[int] = None):
        """A context whose fluid comes from device arrays (objects exposing
        data_ptr(): x (n, 3) and v (n, 3) float64, rho (n,) float64, phase
        (n,) int32, all contiguous on the current device; sph_create_device).
        The scene supplies the walls and every parameter; its own fluid
        arrays are not used.  The arrays are copied on the stream, which
        create synchronises, so they may be freed once this returns."""
        self = cls.__new__(cls)
        self.scene = scene
        self.precision = precision
        self.nf, self.nw = int(x.shape[0]), scene.n_wall
        self._xw = np.ascontiguousarray(scene.wall_pos, np.float64).reshape(-1, 3)
        self.params = make_params(scene, precision)
        dp = lambda a: None if a is None else a.data_ptr()  # noqa: E731
        fluid = sph_fluid(self.nf, dp(x), dp(v), dp(rho), dp(phase))
        wall = sph_wall(self.nw, _ptr(self._xw))
        self.stream = current_stream_handle() if stream is None else stream
        st, ctx = sph_create_device(self.params, fluid, wall, self.stream)
        _check(st, None)
        self.ctx = ctx
        return self

    def close(self):
        if getattr(self, "ctx", None):
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n: int = 1, dt: float = 0.0) -> float:
        st, last = sph_step(self.ctx, n, dt)
        _check(st, self.ctx)
        return last

    def step_async(self, n: int = 1, dt: float = 0.0):
        """Enqueue n steps without waiting (see sph_step_async)."""
        _check(sph_step_async(self.ctx, n, dt), self.ctx)

    def sync(self) -> float:
        st, last = sph_sync(self.ctx)
        _check(st, self.ctx)
        return last

    def reinit_density(self):
        _check(sph_reinit_density(self.ctx), self.ctx)

    def set_excitation(self, amp, freq: float):
        """Rigid tank motion x = amp sin(2 pi freq t) (sph_set_excitation)."""
        a = np.ascontiguousarray(amp, np.float64)
        _check(lib().sph_set_excitation(self.ctx, _ptr(a), float(freq)), self.ctx)

    @property
    def time(self) -> float:
        t = C.c_double(0.0)
        _check(lib().sph_time(self.ctx, C.byref(t)), self.ctx)
        return t.value

    def probe_pressure(self, pts):
        """(p, w) at the points pts (n x 3): the Shepard-interpolated fluid
        pressure and the kernel sum (sph_probe_pressure)."""
        q = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        p, w = np.zeros(len(q)), np.zeros(len(q))
        _check(sph_probe_pressure(self.ctx, _ptr(q), len(q), _ptr(p), _ptr(w)), self.ctx)
        return p, w

    def gauge_height(self, gauges, dz: Optional[float] = None):
        """Free-surface height of the first phase on each vertical line
        (x, y, z_lo, z_hi) of gauges (n x 4), sampled dz apart (default
        dx/4) (sph_gauge_height)."""
        g = np.ascontiguousarray(gauges, np.float64).reshape(-1, 4)
        H = np.zeros(len(g))
        step = 0.25 * self.scene.dp if dz is None else float(dz)
        _check(sph_gauge_height(self.ctx, _ptr(g), len(g), step, _ptr(H)), self.ctx)
        return H

    def state(self) -> dict:
        n, m = self.nf, self.nw
        o = {"x": np.zeros((n, 3)), "v": np.zeros((n, 3)), "rho": np.zeros(n),
             "p": np.zeros(n), "a": np.zeros((n, 3)), "drho_dt": np.zeros(n),
             "sigma": np.zeros(n), "pw": np.zeros(m), "rhow": np.zeros((m, 2)),
             "normal": np.zeros((m, 3))}
        out = sph_state_out(*(_ptr(o[k]) for k in ("x", "v", "rho", "p", "a", "drho_dt",
                                                    "sigma", "pw", "rhow", "normal")))
        _check(sph_get_state(self.ctx, out, SPH_HOST), self.ctx)
        return o

    def grid(self):
        st, dims, nc, cs = sph_grid_info(self.ctx)
        _check(st, self.ctx)
        return dims, nc, cs

    def cells(self) -> dict:
        dims, nc, cs = self.grid()
        o = {"dims": dims, "n_cells": nc,
             "key_f": np.zeros(self.nf, np.uint32), "order_f": np.zeros(self.nf, np.int32),
             "start_f": np.zeros(nc + 1, np.int32), "key_w": np.zeros(self.nw, np.uint32),
             "order_w": np.zeros(self.nw, np.int32), "start_w": np.zeros(nc + 1, np.int32)}
        _check(sph_get_cells(self.ctx, o["key_f"], o["order_f"], o["start_f"], o["key_w"],
                             o["order_w"], o["start_w"]), self.ctx)
        return o

    def neighbors(self) -> dict:
        """The neighbour sets the last step's sweeps visited (sph_get_neighbors):
        CSR arrays in original ids, each particle's ids ascending, and the
        number of particles whose fluid / wall lists overflowed."""
        n = self.nf
        f_off, w_off = np.zeros(n + 1, np.int64), np.zeros(n + 1, np.int64)
        ovf = np.zeros(2, np.int64)
        _check(sph_get_neighbors(self.ctx, f_off, None, 0, w_off, None, 0, ovf), self.ctx)
        f_ids = np.zeros(max(int(f_off[-1]), 1), np.int32)
        w_ids = np.zeros(max(int(w_off[-1]), 1), np.int32)
        _check(sph_get_neighbors(self.ctx, f_off, f_ids, len(f_ids), w_off, w_ids, len(w_ids), ovf),
               self.ctx)
        return {"f_off": f_off, "f_ids": f_ids[:f_off[-1]], "w_off": w_off, "w_ids": w_ids[:w_off[-1]],
                "overflow": ovf}

    def neighbor_totals(self):
        """(fluid-fluid, fluid-wall) ordered pair counts of the last build: the
        totals of sph_get_neighbors, without the ids."""
        n = self.nf
        f_off, w_off = np.zeros(n + 1, np.int64), np.zeros(n + 1, np.int64)
        _check(sph_get_neighbors(self.ctx, f_off, None, 0, w_off, None, 0, None), self.ctx)
        return int(f_off[-1]), int(w_off[-1])

    def neighbor_overflow(self):
        """(fluid, wall): the number of fluid particles whose fluid / wall list
        of the last build overflowed (their sweeps scan the cells)."""
        n = self.nf
        f_off, w_off = np.zeros(n + 1, np.int64), np.zeros(n + 1, np.int64)
        ovf = np.zeros(2, np.int64)
        _check(sph_get_neighbors(self.ctx, f_off, None, 0, w_off, None, 0, ovf), self.ctx)
        return int(ovf[0]), int(ovf[1])

    def diagnostics(self) -> np.ndarray:
        out = np.zeros(8)
        _check(sph_diagnostics(self.ctx, out), self.ctx)
        return out

    def counters(self):
        st, steps, active = sph_counters(self.ctx)
        _check(st, self.ctx)
        return steps, active

    def profile(self, kinds=()):
        """Time the named kernel kinds (see KERNEL_KINDS) from now on."""
        mask = 0
        for k in kinds:
            mask |= 1 << KERNEL_KINDS.index(k)
        _check(sph_profile(self.ctx, mask), self.ctx)

    def profile_read(self) -> dict:
        st, ms, timed, launches = sph_profile_read(self.ctx)
        _check(st, self.ctx)
        return {k: {"ms": float(ms[i]), "timed": int(timed[i]), "launches": int(launches[i])}
                for i, k in enumerate(KERNEL_KINDS)}

    def tape_budget(self, nbytes: int):
        """Device memory the tape may keep step products in (sph_tape_budget;
        -1 = half the free memory, 0 = recompute every step)."""
        _check(lib().sph_tape_budget(self.ctx, int(nbytes)), self.ctx)

    def tape(self, n: int = 1, dt: float = 0.0) -> float:
        """Advance n steps recording checkpoints for backward()."""
        st, last = sph_tape(self.ctx, n, dt)
        _check(st, self.ctx)
        return last

    def backward(self, seed: dict) -> dict:
        """Gradients of L = sum(seed_x.x_N) + sum(seed_v.v_N) + sum(seed_rho rho_N)
        + sum(seed_pw p_w,N) with respect to the created state (x0, v0, rho0)
        and (c0, gamma_p, mu).  Host arrays in original particle order."""
        keep = {k: None if seed.get(k) is None else np.ascontiguousarray(seed[k], np.float64)
                for k in ("x", "v", "rho", "pw")}
        s = sph_adjoint_seed(*(_ptr(keep[k]) for k in ("x", "v", "rho", "pw")))
        out = {"x": np.zeros((self.nf, 3)), "v": np.zeros((self.nf, 3)), "rho": np.zeros(self.nf)}
        g = sph_adjoint_grad(_ptr(out["x"]), _ptr(out["v"]), _ptr(out["rho"]))
        _check(sph_backward(self.ctx, s, g, SPH_HOST), self.ctx)
        out["c0"], out["gamma_p"], out["mu"] = (float(g.params[k]) for k in range(3))
        return out
