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
