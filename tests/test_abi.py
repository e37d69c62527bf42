"""The C-ABI library loads without a GPU and exports exactly what include/damas.h declares,
and the Python binding's ctypes layouts match the C compiler's."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1608_05179_gb300 import _lib
from paper_1608_05179_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "damas.h")


def _declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, flags=re.M))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    decl = _declared_functions()
    assert {"damas_build_psf", "das_map", "wavelet_compress_grid", "damas_solve"} <= decl
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = decl - exported
    assert not missing, missing
    assert decl == set(_lib.SIGNATURES), decl ^ set(_lib.SIGNATURES)
    for name in decl:
        assert getattr(lib, name) is not None


def test_struct_layouts_match_c():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "damas.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(damas_geom), sizeof(damas_wavelet_cfg), sizeof(damas_system), sizeof(damas_solve_cfg));
  printf("%zu %zu %zu %zu\n", offsetof(damas_geom, formulation), offsetof(damas_system, ctas), offsetof(damas_solve_cfg, a_placement), offsetof(damas_geom, diag_removal));
  printf("%zu %zu %zu %zu\n", sizeof(damas_result), offsetof(damas_result, t_solve), offsetof(damas_result, hbm_bytes), offsetof(damas_result, sm_units));
  printf("%zu %zu %zu\n", sizeof(damas_request), sizeof(damas_serve_cfg), offsetof(damas_request, iters));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        l1, l2, l3, l4 = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")[:4]
    sizes = [int(v) for v in l1.split()]
    offs = [int(v) for v in l2.split()]
    assert sizes == [ctypes.sizeof(_lib.damas_geom), ctypes.sizeof(_lib.damas_wavelet_cfg),
                     ctypes.sizeof(_lib.damas_system), ctypes.sizeof(_lib.damas_solve_cfg)]
    assert offs == [_lib.damas_geom.formulation.offset, _lib.damas_system.ctas.offset,
                    _lib.damas_solve_cfg.a_placement.offset, _lib.damas_geom.diag_removal.offset]
    assert [int(v) for v in l3.split()] == [ctypes.sizeof(_lib.damas_result), _lib.damas_result.t_solve.offset,
                                            _lib.damas_result.hbm_bytes.offset, _lib.damas_result.sm_units.offset]
    assert [int(v) for v in l4.split()] == [ctypes.sizeof(_lib.damas_request), ctypes.sizeof(_lib.damas_serve_cfg),
                                            _lib.damas_request.iters.offset]


def test_host_only_entry_points(lib):
    assert lib.damas_lda(1) == 32 and lib.damas_lda(33) == 64 and lib.damas_lda(657) == 672
    assert lib.damas_lda(0) == 0
    assert lib.damas_state_floats(100) == 264 and lib.damas_state_floats(0) == 0


def test_create_rejects_bad_device(lib):
    h = ctypes.c_void_p()
    assert lib.damas_create(ctypes.byref(h), -1) == _lib.DAMAS_EINVAL
    assert lib.damas_create(ctypes.byref(h), 1 << 20) == _lib.DAMAS_EINVAL
    assert not h.value


def test_null_context_is_rejected(lib):
    assert lib.damas_destroy(None) == _lib.DAMAS_EINVAL
    assert lib.damas_solve(None, None, 0, None, None) == _lib.DAMAS_EINVAL
