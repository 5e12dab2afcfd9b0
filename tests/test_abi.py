"""CPU-side checks of the C ABI: the library builds, loads and exports every
function include/dg.h declares; the binding and header agree on struct sizes.
No compute call is made (there may be no GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_06841_gb300 import build
    build.build()
    return C.CDLL(build.OUT)


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("dg_init", "dg_rhs", "dg_step", "dg_set_forcing", "dg_diagnostics"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    from paper_2401_06841_gb300 import _lib as B
    assert sorted(B.EXPORTS) == declared_functions()


def test_struct_sizes_match_header():
    # compile a tiny C program against the header and compare sizeof()s
    import subprocess
    import tempfile
    from paper_2401_06841_gb300 import _lib as B
    prog = r'''
#include <stdio.h>
#include "dg.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dg_mesh), sizeof(dg_nu_params), sizeof(dg_opts),
 sizeof(dg_forcing), sizeof(dg_diag), sizeof(dg_meta), sizeof(dg_prof), sizeof(dg_adi_opts)); return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    mine = [C.sizeof(B.Mesh), C.sizeof(B.NuParams), C.sizeof(B.Opts), C.sizeof(B.Forcing), C.sizeof(B.Diag),
            C.sizeof(B.Meta), C.sizeof(B.Prof), C.sizeof(B.AdiOpts)]
    assert sizes == mine


def test_scratch_query_and_argument_validation(lib):
    # pure host paths: no device is touched
    from paper_2401_06841_gb300 import _lib as B
    L = B.lib()
    mesh = B.Mesh((C.c_int32 * 3)(8, 8, 8), (C.c_double * 3)(1, 1, 1))
    nu = B.NuParams(1, 2.0, 0.2, 1e-3, 0.0)
    n = C.c_size_t(0)
    assert L.dg_scratch_bytes(C.byref(mesh), 3, C.byref(nu), C.byref(n)) == 0 and n.value > 0
    assert L.dg_scratch_bytes(C.byref(mesh), 7, C.byref(nu), C.byref(n)) == B.DG_EINVAL
    h = C.c_void_p(0)
    opts = B.Opts()
    assert L.dg_init(C.byref(h), C.byref(mesh), 3, 1.0, C.byref(nu), C.byref(opts)) == B.DG_EINVAL
    assert not h.value
    bad = B.Mesh((C.c_int32 * 3)(8, 8, 4), (C.c_double * 3)(1, 1, 1))
    assert L.dg_init(C.byref(h), C.byref(bad), 3, 1.0, C.byref(nu), C.byref(opts)) == B.DG_EINVAL
    assert L.dg_step(None, 1, 0.0, None, None) == B.DG_EINVAL
    assert L.dg_rhs(None, None, None, None, 0.0) == B.DG_EINVAL
