"""Plain FP64 CPU oracle of the WCSPH step (arXiv 2110.02621), via ctypes.

TEST INFRASTRUCTURE ONLY.  The oracle checks the CUDA library and is never
part of it: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA path; both take their inputs from ``paper_2110_02621_gb300.scenes``.

The C source (``sph_oracle.c``) follows the paper's equations one by one; see
its header for the readings taken where the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_sph.so")

EOS = {"linear": 0, "tait": 1}
DENSITY = {"continuity": 0, "summation": 1}
REINIT = {"none": 0, "free_surface": 1, "internal": 2}


def compile_command(src: str, out: str) -> list:
    """The gcc command that builds the oracle library from src."""
    return ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
            "-shared", "-o", out, src, "-lm"]


# A prebuilt library to load instead (the mutation tests load deliberately
# broken copies of the oracle this way, in subprocesses of their own).
_LIB_OVERRIDE = "SPH_ORACLE_LIB"


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, FP64, no contraction)."""
    if os.environ.get(_LIB_OVERRIDE):
        return os.environ[_LIB_OVERRIDE]
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(_SRC[:-1] + "h"))):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(compile_command(_SRC, tmp))
    os.replace(tmp, _LIB)
    return _LIB


class _Phase(C.Structure):
    _fields_ = [("rho0", C.c_double), ("mu", C.c_double), ("z_top", C.c_double),
                ("eos", C.c_int32), ("density", C.c_int32),
                ("reinit", C.c_int32), ("penalty", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("dp", C.c_double), ("h", C.c_double), ("c0", C.c_double),
                ("gamma_tait", C.c_double), ("gamma_p", C.c_double),
                ("cfl", C.c_double), ("g", C.c_double * 3),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("n_phases", C.c_int32), ("reinit_every", C.c_int32),
                ("phase", _Phase * 2), ("dim", C.c_int32), ("periodic", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i32, i64, p = C.c_double, C.c_int32, C.c_int64, C.c_void_p
        sig = {
            "orc_W": (d, [d, d]), "orc_dWdr": (d, [d, d]),
            "orc_W_dim": (d, [d, d, i32]), "orc_dWdr_dim": (d, [d, d, i32]),
            "orc_lattice_sigma0_dim": (d, [d, d, i32]),
            "orc_eos_p": (d, [d, p, d, d]), "orc_eos_rho": (d, [d, p, d, d]),
            "orc_riemann": (None, [d, d, d, d, d, d, d, i32, p]),
            "orc_lattice_sigma0": (d, [d, d]),
            "orc_create": (p, [p, i64, p, p, p, p, i64, p]),
            "orc_destroy": (None, [p]), "orc_step": (d, [p, i32, d]),
            "orc_reinit_density": (None, [p]), "orc_rates": (None, [p, p, p]),
            "orc_get_fluid": (None, [p] * 8), "orc_get_wall": (None, [p] * 4),
            "orc_n_cells": (i64, [p, p]), "orc_get_cells": (None, [p] * 7),
            "orc_neighbors": (i64, [p, i64, p, i64, p, p, i64, p]),
            "orc_diagnostics": (None, [p, p]), "orc_sigma0": (d, [p]),
            "orc_step_count": (i64, [p]), "orc_threads": (i32, []),
            "orc_set_threads": (None, [i32]),
            "orc_set_excitation": (None, [p, p, d]), "orc_time": (d, [p]),
            "orc_probe_pressure": (None, [p, p, i64, p, p]),
            "orc_gauge_height": (None, [p, p, i64, d, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_phase(ph) -> _Phase:
    return _Phase(rho0=ph.rho0, mu=ph.mu, z_top=ph.z_top, eos=EOS[ph.eos],
                  density=DENSITY[ph.density], reinit=REINIT[ph.reinit],
                  penalty=int(bool(ph.penalty)))


def make_params(scene) -> _Params:
    P = _Params()
    P.dp, P.h, P.c0 = scene.dp, scene.h, scene.c0
    P.gamma_tait, P.gamma_p, P.cfl = scene.gamma_tait, scene.gamma_p, scene.cfl
    for d in range(3):
        P.g[d], P.lo[d], P.hi[d] = scene.g[d], scene.lo[d], scene.hi[d]
    P.n_phases = len(scene.phases)
    P.reinit_every = scene.reinit_every
    P.dim = getattr(scene, "dim", 3)
    per = getattr(scene, "periodic", (0, 0, 0))
    P.periodic = sum(1 << d for d in range(3) if per[d])
    for k, ph in enumerate(scene.phases):
        P.phase[k] = make_phase(ph)
    return P


def W(r: float, h: float, dim: int = 3) -> float:
    return lib().orc_W(r, h) if dim == 3 else lib().orc_W_dim(r, h, dim)


def dWdr(r: float, h: float, dim: int = 3) -> float:
    return lib().orc_dWdr(r, h) if dim == 3 else lib().orc_dWdr_dim(r, h, dim)


def eos_p(rho: float, phase, c0: float, gamma_tait: float = 7.0) -> float:
    ph = make_phase(phase)
    return lib().orc_eos_p(rho, C.byref(ph), c0, gamma_tait)


def eos_rho(p: float, phase, c0: float, gamma_tait: float = 7.0) -> float:
    ph = make_phase(phase)
    return lib().orc_eos_rho(p, C.byref(ph), c0, gamma_tait)


def riemann(rhoL, UL, pL, rhoR, UR, pR, c, limiter=True):
    """Returns (U*, p*, U_bar, P_bar) of Eq. (RSsolution)."""
    out = np.zeros(4)
    lib().orc_riemann(rhoL, UL, pL, rhoR, UR, pR, c, int(limiter), _ptr(out))
    return tuple(out)


def lattice_sigma0(dp: float, h: float, dim: int = 3) -> float:
    return lib().orc_lattice_sigma0(dp, h) if dim == 3 else lib().orc_lattice_sigma0_dim(dp, h, dim)


def set_threads(n: int):
    """OpenMP threads the oracle uses from now on."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    return lib().orc_threads()


class OracleSim:
    """FP64 simulation of a scene, state kept in original particle order."""

    def __init__(self, scene, rho: Optional[np.ndarray] = None):
        L = lib()
        self.scene = scene
        self.params = make_params(scene)
        self.nf, self.nw = scene.n_fluid, scene.n_wall
        x = np.ascontiguousarray(scene.fluid_pos, np.float64)
        v = np.ascontiguousarray(scene.fluid_vel, np.float64)
        ph = np.ascontiguousarray(scene.fluid_phase, np.int32)
        xw = np.ascontiguousarray(scene.wall_pos, np.float64).reshape(-1, 3)
        if rho is None:
            rho = getattr(scene, "rho_init", None)
        r = None if rho is None else np.ascontiguousarray(rho, np.float64)
        self._h = L.orc_create(C.byref(self.params), self.nf, _ptr(x), _ptr(v),
                               _ptr(r), _ptr(ph), self.nw, _ptr(xw))
        if not self._h:
            raise RuntimeError("orc_create failed")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1, dt: float = 0.0) -> float:
        return lib().orc_step(self._h, int(n), float(dt))

    def reinit_density(self):
        lib().orc_reinit_density(self._h)

    def set_excitation(self, amp, freq: float):
        """Rigid sinusoidal tank motion x = amp sin(2 pi freq t), in the tank frame."""
        a = np.ascontiguousarray(amp, np.float64)
        lib().orc_set_excitation(self._h, _ptr(a), float(freq))

    @property
    def time(self) -> float:
        return lib().orc_time(self._h)

    def rates(self):
        drho = np.zeros(self.nf)
        a = np.zeros((self.nf, 3))
        lib().orc_rates(self._h, _ptr(drho), _ptr(a))
        return drho, a

    def fluid(self) -> dict:
        n = self.nf
        out = {k: np.zeros((n, 3)) for k in ("x", "v", "a")}
        out.update({k: np.zeros(n) for k in ("rho", "p", "drho_dt", "sigma")})
        lib().orc_get_fluid(self._h, _ptr(out["x"]), _ptr(out["v"]),
                            _ptr(out["rho"]), _ptr(out["p"]), _ptr(out["a"]),
                            _ptr(out["drho_dt"]), _ptr(out["sigma"]))
        return out

    def wall(self) -> dict:
        n = self.nw
        out = {"pw": np.zeros(n), "rhow": np.zeros((n, 2)),
               "normal": np.zeros((n, 3))}
        lib().orc_get_wall(self._h, _ptr(out["pw"]), _ptr(out["rhow"]),
                           _ptr(out["normal"]))
        return out

    def cells(self) -> dict:
        dims = np.zeros(3, np.int32)
        nc = lib().orc_n_cells(self._h, _ptr(dims))
        out = {"dims": dims, "n_cells": int(nc),
               "key_f": np.zeros(self.nf, np.uint32),
               "order_f": np.zeros(self.nf, np.int64),
               "start_f": np.zeros(nc + 1, np.int64),
               "key_w": np.zeros(self.nw, np.uint32),
               "order_w": np.zeros(self.nw, np.int64),
               "start_w": np.zeros(nc + 1, np.int64)}
        lib().orc_get_cells(self._h, *(_ptr(out[k]) for k in
                                       ("key_f", "order_f", "start_f", "key_w",
                                        "order_w", "start_w")))
        return out

    def neighbors(self, i: int, max_n: int = 4096):
        f = np.zeros(max_n, np.int64)
        w = np.zeros(max_n, np.int64)
        nf, nw = C.c_int64(), C.c_int64()
        lib().orc_neighbors(self._h, int(i), _ptr(f), max_n, C.byref(nf),
                            _ptr(w), max_n, C.byref(nw))
        return f[:nf.value].copy(), w[:nw.value].copy()

    def diagnostics(self) -> np.ndarray:
        out = np.zeros(8)
        lib().orc_diagnostics(self._h, _ptr(out))
        return out

    def probe_pressure(self, pts):
        """(p_bar, w) at the points pts (n x 3): Shepard-interpolated pressure
        and kernel sum over the fluid particles (Sec. 4.3 sensors)."""
        q = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
        p, w = np.zeros(len(q)), np.zeros(len(q))
        lib().orc_probe_pressure(self._h, _ptr(q), len(q), _ptr(p), _ptr(w))
        return p, w

    def gauge_height(self, gauges, dz: float):
        """Free-surface height on each vertical line (x, y, z_lo, z_hi) of
        gauges (n x 4), sampled dz apart (Sec. 4.3 wave gauges)."""
        g = np.ascontiguousarray(gauges, np.float64).reshape(-1, 4)
        H = np.zeros(len(g))
        lib().orc_gauge_height(self._h, _ptr(g), len(g), float(dz), _ptr(H))
        return H

    @property
    def sigma0(self) -> float:
        return lib().orc_sigma0(self._h)

    @property
    def step_count(self) -> int:
        return lib().orc_step_count(self._h)
