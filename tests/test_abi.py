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
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dg_mesh), sizeof(dg_nu_params), sizeof(dg_opts),
 sizeof(dg_forcing), sizeof(dg_diag), sizeof(dg_meta), sizeof(dg_prof), sizeof(dg_adi_opts), sizeof(dg_adi_meta));
 return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe]).split()]
    mine = [C.sizeof(B.Mesh), C.sizeof(B.NuParams), C.sizeof(B.Opts), C.sizeof(B.Forcing), C.sizeof(B.Diag),
            C.sizeof(B.Meta), C.sizeof(B.Prof), C.sizeof(B.AdiOpts), C.sizeof(B.AdiMeta)]
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
    # the size queries reject the meshes dg_init rejects: too fine, empty, not cubic
    for dims in ((1025, 1025, 1025), (0, 0, 0), (8, 8, 4)):
        m = B.Mesh((C.c_int32 * 3)(*dims), (C.c_double * 3)(1, 1, 1))
        assert L.dg_scratch_bytes(C.byref(m), 3, C.byref(nu), C.byref(n)) == B.DG_EINVAL, dims
        assert L.dg_vhat_bytes(C.byref(m), 3, 0, C.byref(n)) == B.DG_EINVAL, dims
    top = B.Mesh((C.c_int32 * 3)(1024, 1024, 1024), (C.c_double * 3)(1, 1, 1))
    assert L.dg_scratch_bytes(C.byref(top), 3, C.byref(nu), C.byref(n)) == 0 and n.value > 0
    h = C.c_void_p(0)
    opts = B.Opts()
    assert L.dg_init(C.byref(h), C.byref(mesh), 3, 1.0, C.byref(nu), C.byref(opts)) == B.DG_EINVAL
    assert not h.value
    bad = B.Mesh((C.c_int32 * 3)(8, 8, 4), (C.c_double * 3)(1, 1, 1))
    assert L.dg_init(C.byref(h), C.byref(bad), 3, 1.0, C.byref(nu), C.byref(opts)) == B.DG_EINVAL
    assert L.dg_step(None, 1, 0.0, None, None) == B.DG_EINVAL
    assert L.dg_rhs(None, None, None, None, 0.0) == B.DG_EINVAL


def test_adiabatic_buffer_sizes_and_argument_validation(lib):
    # host-only paths of the dg_adi_* entry points: no device is touched
    from paper_2401_06841_gb300 import _lib as B
    L = B.lib()
    sz = [C.c_size_t(0) for _ in range(3)]
    N, k = 8, 3
    b = (k + 1) * (k + 2) * (k + 3) // 6
    mesh = B.Mesh((C.c_int32 * 3)(N, N, N), (C.c_double * 3)(1, 1, 1))
    for prec, el in ((B.PREC_F32, 4), (B.PREC_F64, 8)):
        assert L.dg_adi_buffer_bytes(C.byref(mesh), k, prec, *[C.byref(x) for x in sz]) == 0
        assert sz[0].value == N ** 3 * 5 * b * el  # state register
        assert sz[1].value == N ** 3 * 4 * b * el  # projections of v and p
        # scratch: the second projection buffer and the driving a_h plus fixed parts
        assert sz[2].value > N ** 3 * 7 * b * el
    assert L.dg_adi_buffer_bytes(C.byref(mesh), k, B.PREC_X3, *[C.byref(x) for x in sz]) == B.DG_EINVAL
    assert L.dg_adi_buffer_bytes(C.byref(mesh), 4, B.PREC_F32, *[C.byref(x) for x in sz]) == B.DG_EINVAL
    big = B.Mesh((C.c_int32 * 3)(1025, 1025, 1025), (C.c_double * 3)(1, 1, 1))
    assert L.dg_adi_buffer_bytes(C.byref(big), k, B.PREC_F32, *[C.byref(x) for x in sz]) == B.DG_EINVAL
    flat = B.Mesh((C.c_int32 * 3)(8, 8, 4), (C.c_double * 3)(1, 1, 1))
    assert L.dg_adi_buffer_bytes(C.byref(flat), k, B.PREC_F32, *[C.byref(x) for x in sz]) == B.DG_EINVAL
    h = C.c_void_p(0)
    nu = B.NuParams(1, 2.0, 0.2, 1e-3, 0.0, 0.0, 0)
    opts = B.AdiOpts()  # null buffers, gamma 0: rejected before any device call
    assert L.dg_adi_init(C.byref(h), C.byref(mesh), k, C.byref(nu), C.byref(opts)) == B.DG_EINVAL
    assert not h.value
    learned = B.NuParams(2, 2.0, 0.2, 1e-3, 0.0, 0.0, 0)
    assert L.dg_adi_init(C.byref(h), C.byref(mesh), k, C.byref(learned), C.byref(opts)) == B.DG_EINVAL
    assert L.dg_adi_step(None, 1, 0.0, None, None) == B.DG_EINVAL
    assert L.dg_adi_rhs(None, None, None, 0.0) == B.DG_EINVAL
    assert L.dg_adi_set_reset(None, 1.0) == B.DG_EINVAL
    assert L.dg_adi_energy_budget(None, None) == B.DG_EINVAL


def test_a_c_program_links_and_queries_sizes(lib):
    # the header's prototypes used from C itself, linked against libdg.so:
    # the size queries (no device touched) agree with the ctypes binding and
    # reject the meshes the constructors reject
    import shutil
    import subprocess
    import tempfile
    from paper_2401_06841_gb300 import _lib as B
    from paper_2401_06841_gb300 import build
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    prog = r'''
#include <stdio.h>
#include "dg.h"
int main(void) {
    dg_mesh m = {{64, 64, 64}, {1.0, 1.0, 1.0}}, bad = {{64, 64, 32}, {1.0, 1.0, 1.0}};
    dg_nu_params nu = {0};
    size_t s = 0, v = 0, us = 0, up = 0, usc = 0;
    nu.mode = DG_AV_LEARNED;
    int r1 = dg_scratch_bytes(&m, 3, &nu, &s);
    int r2 = dg_vhat_bytes(&m, 3, DG_PREC_X3, &v);
    int r3 = dg_adi_buffer_bytes(&m, 3, DG_PREC_F32, &us, &up, &usc);
    int r4 = dg_scratch_bytes(&bad, 3, &nu, &s);
    printf("%d %d %d %d %zu %zu %zu %zu %zu\n", r1, r2, r3, r4, s, v, us, up, usc);
    return 0;
}
'''
    pkg = os.path.dirname(build.OUT)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "q.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "q")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe, "-L", pkg, "-ldg",
                               "-Wl,-rpath," + pkg, "-L/usr/local/cuda/lib64", "-Wl,-rpath-link,/usr/local/cuda/lib64"])
        out = subprocess.check_output([exe]).split()
    r1, r2, r3, r4, s, v, us, up, usc = [int(x) for x in out]
    assert (r1, r2, r3) == (0, 0, 0) and r4 == B.DG_EINVAL
    L = B.lib()
    mesh = B.Mesh((C.c_int32 * 3)(64, 64, 64), (C.c_double * 3)(1, 1, 1))
    nu = B.NuParams(B.AV_LEARNED, 0.0, 0.0, 0.0, 0.0)
    n = C.c_size_t(0)
    assert L.dg_scratch_bytes(C.byref(mesh), 3, C.byref(nu), C.byref(n)) == 0 and n.value == s
    assert L.dg_vhat_bytes(C.byref(mesh), 3, B.PREC_X3, C.byref(n)) == 0 and n.value == v
    sz = [C.c_size_t(0) for _ in range(3)]
    assert L.dg_adi_buffer_bytes(C.byref(mesh), 3, B.PREC_F32, *[C.byref(x) for x in sz]) == 0
    assert [x.value for x in sz] == [us, up, usc]
    b = 20
    assert us == 64 ** 3 * 5 * b * 4 and up == 64 ** 3 * 4 * b * 4


def test_c_example_compiles_and_links(lib):
    # the C example of the ABI (tests/c/run_ten_steps.c) against the header,
    # libdg.so and the CUDA runtime (compiled and linked only: running it needs a GPU)
    import shutil
    import subprocess
    import tempfile
    from paper_2401_06841_gb300 import build
    if shutil.which("gcc") is None or not os.path.isdir("/usr/local/cuda/include"):
        pytest.skip("no C compiler or CUDA headers")
    src = open(os.path.join(ROOT, "tests", "c", "run_ten_steps.c")).read()
    pkg = os.path.dirname(build.OUT)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "example.c")
        open(c, "w").write(src + "\nint main(void) { return 0; }\n")
        subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                               "-I", "/usr/local/cuda/include", c, "-o", os.path.join(d, "example"),
                               "-L", pkg, "-ldg", "-Wl,-rpath," + pkg, "-L/usr/local/cuda/lib64", "-lcudart"])
