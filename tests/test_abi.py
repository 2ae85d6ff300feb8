"""The C ABI without a GPU: the library loads, exports every function that
include/sph.h declares, and the ctypes structures match the header's layout
as gcc compiles it."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2110_02621_gb300 import build, sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sph.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(sph.EXPORTS)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "sph.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(sph_phase), sizeof(sph_params), sizeof(sph_fluid),
         sizeof(sph_wall), sizeof(sph_state_out));
  printf("%zu %zu %zu %zu\n", offsetof(sph_params, phase), offsetof(sph_params, precision),
         offsetof(sph_params, n_phases), offsetof(sph_state_out, normal));
  printf("%zu %zu %zu\n", sizeof(sph_adjoint_seed), sizeof(sph_adjoint_grad),
         offsetof(sph_adjoint_grad, params));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    sizes, offs, adj = subprocess.check_output([str(exe)]).decode().split("\n")[:3]
    assert [int(v) for v in sizes.split()] == [C.sizeof(sph.sph_phase), C.sizeof(sph.sph_params),
                                               C.sizeof(sph.sph_fluid), C.sizeof(sph.sph_wall),
                                               C.sizeof(sph.sph_state_out)]
    assert [int(v) for v in offs.split()] == [sph.sph_params.phase.offset, sph.sph_params.precision.offset,
                                              sph.sph_params.n_phases.offset, sph.sph_state_out.normal.offset]
    assert [int(v) for v in adj.split()] == [C.sizeof(sph.sph_adjoint_seed), C.sizeof(sph.sph_adjoint_grad),
                                             sph.sph_adjoint_grad.params.offset]


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    """Validation runs before any CUDA call, so these return SPH_ERR_ARG here."""
    from paper_2110_02621_gb300 import scenes
    sc = scenes.still_water_tank(n_fluid=(3, 3, 3))
    P = sph.make_params(sc)
    x = sc.fluid_pos.copy()
    F = sph.sph_fluid(len(x), x.ctypes.data, None, None, None)
    bad = sph.make_params(sc)
    bad.h = -1.0
    st, ctx = sph.sph_create(bad, F, None)
    assert st == sph.SPH_ERR_ARG and not ctx.value
    assert "h" in sph.sph_last_error(None)
    bad = sph.make_params(sc)
    bad.n_phases = 3
    assert sph.sph_create(bad, F, None)[0] == sph.SPH_ERR_ARG
    ph = (sc.fluid_phase + 1).astype("int32")
    F2 = sph.sph_fluid(len(x), x.ctypes.data, None, None, ph.ctypes.data)
    assert sph.sph_create(P, F2, None)[0] == sph.SPH_ERR_ARG
    xn = x.copy()
    xn[0, 0] = float("nan")
    F3 = sph.sph_fluid(len(x), xn.ctypes.data, None, None, None)
    assert sph.sph_create(P, F3, None)[0] == sph.SPH_ERR_ARG
    assert lib.sph_step(None, 1, 0.0, None) == sph.SPH_ERR_ARG
    lib.sph_destroy(None)


def _p_set(**kw):
    def f(P, F, W, keep):
        for k, v in kw.items():
            setattr(P, k, v)
    return f


def _phase_set(**kw):
    def f(P, F, W, keep):
        for k, v in kw.items():
            setattr(P.phase[0], k, v)
    return f


def _axis(field, d, value):
    def f(P, F, W, keep):
        getattr(P, field)[d] = value
    return f


def _fluid_array(name, value, row=0, col=0):
    def f(P, F, W, keep):
        import numpy as np
        a = np.array(keep[name], dtype=keep[name].dtype, copy=True)
        if a.ndim == 2:
            a[row, col] = value
        else:
            a[row] = value
        keep[name + "_bad"] = a
        setattr(F, name, a.ctypes.data)
    return f


def _periodic_box_axis(P, F, W, keep):
    P.periodic = 1
    P.hi[0] = P.lo[0] + 2 * P.h * 4.3  # 4.3 cells: not whole


def _tiny_cells(P, F, W, keep):
    P.h = 1e-4  # 2h cells of 0.2 mm over a 0.1 m box: ~1.3e8 cells


def _two_d_periodic_y(P, F, W, keep):
    P.dim = 2
    P.periodic = 2


REJECTIONS = [
    ("h <= 0", _p_set(h=-1.0), "must be finite and > 0"),
    ("c0 = 0", _p_set(c0=0.0), "must be finite and > 0"),
    ("cfl nan", _p_set(cfl=float("nan")), "must be finite and > 0"),
    ("gamma_p < 0", _p_set(gamma_p=-0.1), "gamma_p >= 0"),
    ("g inf", _axis("g", 2, float("inf")), "g, lo, hi must be finite"),
    ("hi <= lo", _axis("hi", 1, -1.0), "hi must exceed lo"),
    ("n_phases 0", _p_set(n_phases=0), "n_phases must be 1 or 2"),
    ("reinit_every < 0", _p_set(reinit_every=-1), "reinit_every"),
    ("precision", _p_set(precision=7), "unknown precision"),
    ("dim 1", _p_set(dim=1), "dim must be"),
    ("rho0 <= 0", _phase_set(rho0=0.0), "phase rho0"),
    ("mu < 0", _phase_set(mu=-1.0), "phase rho0"),
    ("eos 2", _phase_set(eos=2), "out of range"),
    ("reinit 3", _phase_set(reinit=3), "out of range"),
    ("periodic mask", _p_set(periodic=8), "periodic is a mask"),
    ("2-D periodic y", _two_d_periodic_y, "y cannot be periodic"),
    ("fractional period", _periodic_box_axis, "whole number"),
    ("too many cells", _tiny_cells, "too many cells"),
    ("fluid n < 0", lambda P, F, W, keep: setattr(F, "n", -1), "fluid.n"),
    ("fluid n = 2^26", lambda P, F, W, keep: setattr(F, "n", 1 << 26), "fluid.n"),
    ("wall n = 2^26", lambda P, F, W, keep: setattr(W, "n", 1 << 26), "wall.n"),
    ("fluid pos NULL", lambda P, F, W, keep: setattr(F, "pos", None), "fluid.pos"),
    ("wall pos NULL", lambda P, F, W, keep: setattr(W, "pos", None), "wall.pos"),
    ("fluid velocity nan", _fluid_array("vel", float("nan"), 1, 2), "velocity"),
    ("fluid rho <= 0", _fluid_array("rho", 0.0, 2), "rho must be > 0"),
    ("fluid phase out of range", _fluid_array("phase", 1, 3), "phase out of range"),
]


@pytest.mark.parametrize("what,spoil,message", REJECTIONS, ids=[r[0] for r in REJECTIONS])
def test_each_validation_rule_refuses_before_any_cuda_call(lib, what, spoil, message):
    """Every rule of sph_create's validation returns SPH_ERR_ARG with its own
    message, no context, and no CUDA call (so it runs here, without a GPU)."""
    import numpy as np
    from paper_2110_02621_gb300 import scenes
    sc = scenes.still_water_tank(n_fluid=(3, 3, 3))
    P = sph.make_params(sc)
    keep = {"pos": np.ascontiguousarray(sc.fluid_pos), "vel": np.zeros((sc.n_fluid, 3)),
            "rho": np.full(sc.n_fluid, 1000.0), "phase": np.zeros(sc.n_fluid, np.int32),
            "wall": np.ascontiguousarray(sc.wall_pos)}
    F = sph.sph_fluid(sc.n_fluid, keep["pos"].ctypes.data, keep["vel"].ctypes.data, keep["rho"].ctypes.data,
                      keep["phase"].ctypes.data)
    W = sph.sph_wall(len(keep["wall"]), keep["wall"].ctypes.data)
    spoil(P, F, W, keep)
    st, ctx = sph.sph_create(P, F, W)
    assert st == sph.SPH_ERR_ARG and not ctx.value, what
    assert message in sph.sph_last_error(None), (what, sph.sph_last_error(None))


@pytest.mark.parametrize("dims", [(1 << 21, 1 << 21, 1 << 22), (2**31 - 1, 2**31 - 1, 2**31 - 1),
                                  (1 << 12, 1 << 12, 1), (0, 5, 5), (5, -3, 5)],
                         ids=["product_wraps_to_zero", "int32_max_extents", "one_cell_too_many",
                              "zero_extent", "negative_extent"])
@pytest.mark.parametrize("fn", ["sph_bin_sort", "sph_bin_sort_noalloc"])
def test_binning_refuses_grids_beyond_the_scan(lib, fn, dims):
    """A grid of more cells than the scan takes (2^24 - 2), or whose cell count
    would overflow a 64-bit product of the extents (2^21 x 2^21 x 2^22 wraps to
    0), or with an extent below 1, is refused with SPH_ERR_ARG before any
    launch: the pointers below are never dereferenced, so this runs without a
    GPU."""
    dummy = 1 << 20  # never dereferenced: validation comes first
    st = getattr(sph, fn)(dummy, 10, (0.0, 0.0, 0.0), 0.013, dims, dummy, dummy, dummy, 0)
    assert st == sph.SPH_ERR_ARG


DEVICE_SIDE = ("velocity", "rho must be > 0", "phase out of range")


@pytest.mark.parametrize("what,spoil,message", [r for r in REJECTIONS if r[2] not in DEVICE_SIDE],
                         ids=[r[0] for r in REJECTIONS if r[2] not in DEVICE_SIDE])
def test_create_device_refuses_on_the_host_before_any_cuda_call(lib, what, spoil, message):
    """sph_create_device applies the same host-side rules as sph_create
    (everything but the per-particle checks, which it runs on the device) and
    refuses before any CUDA call."""
    import numpy as np
    from paper_2110_02621_gb300 import scenes
    sc = scenes.still_water_tank(n_fluid=(3, 3, 3))
    P = sph.make_params(sc)
    keep = {"pos": np.ascontiguousarray(sc.fluid_pos), "vel": np.zeros((sc.n_fluid, 3)),
            "rho": np.full(sc.n_fluid, 1000.0), "phase": np.zeros(sc.n_fluid, np.int32),
            "wall": np.ascontiguousarray(sc.wall_pos)}
    F = sph.sph_fluid(sc.n_fluid, keep["pos"].ctypes.data, keep["vel"].ctypes.data, keep["rho"].ctypes.data,
                      keep["phase"].ctypes.data)
    W = sph.sph_wall(len(keep["wall"]), keep["wall"].ctypes.data)
    spoil(P, F, W, keep)
    st, ctx = sph.sph_create_device(P, F, W)
    assert st == sph.SPH_ERR_ARG and not ctx.value, what
    assert message in sph.sph_last_error(None), (what, sph.sph_last_error(None))
