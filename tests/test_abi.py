"""Host-side checks of the C interface: the library loads, exports what include/rpa.h
declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rpa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_01816_gb300 as m
    return m


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rpa_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_function(rpa):
    lib = rpa.library()
    names = declared_functions()
    assert {"rpa_setup", "rpa_apply_nuchi0", "rpa_sternheimer_solve", "rpa_coulomb_apply", "rpa_ec"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(rpa.EXPORTED) <= names


def test_default_options_and_version(rpa):
    o = rpa.default_options()
    assert o.prec == rpa.RPA_FP64 and o.tol == 1e-8 and o.n_omega == 8 and o.n_atoms == 1
    assert "sm_103a" in rpa.rpa_version()


def test_struct_layouts_match_header(rpa, tmp_path):
    """The ctypes mirrors of rpa_options / rpa_stats agree with the C compiler's layout."""
    src = tmp_path / "sizes.c"
    src.write_text("""#include <stdio.h>
#include <stddef.h>
#include "rpa.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rpa_options), sizeof(rpa_stats),
         offsetof(rpa_options, independent_frequencies), offsetof(rpa_stats, ms_coulomb),
         offsetof(rpa_stats, worst_status), offsetof(rpa_stats, prof_bytes), offsetof(rpa_stats, launches),
         offsetof(rpa_stats, near_breakdowns), offsetof(rpa_options, sq_order), offsetof(rpa_options, contractions),
         offsetof(rpa_options, periodic), offsetof(rpa_options, precondition), offsetof(rpa_options, block_cocg));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    O, S = rpa.rpa.rpa_options, rpa.rpa.rpa_stats
    assert got == [ctypes.sizeof(O), ctypes.sizeof(S), O.independent_frequencies.offset, S.ms_coulomb.offset,
                   S.worst_status.offset, S.prof_bytes.offset, S.launches.offset,
                   S.near_breakdowns.offset, O.sq_order.offset, O.contractions.offset, O.periodic.offset,
                   O.precondition.offset, O.block_cocg.offset]


def test_setup_rejects_bad_arguments_without_a_gpu(rpa):
    lib = rpa.library()
    hd = ctypes.c_void_p()
    eps = (ctypes.c_double * 1)(-1.0)
    opt = rpa.rpa.rpa_options()
    lib.rpa_default_options(ctypes.byref(opt))
    # zero grid, bad h, bad order, NULL inputs: all rejected by validation
    cases = [(0, 4, 4, 0.5, 12, 1, 1), (4, 4, 4, -1.0, 12, 1, 1), (4, 4, 4, 0.5, 8, 1, 1),
             (4, 4, 4, 0.5, 12, None, 1)]
    for nx, ny, nz, h, order, vl, ps in cases:
        st = lib.rpa_setup(ctypes.byref(hd), nx, ny, nz, h, order, vl, ps, eps, 1, ctypes.byref(opt), None)
        assert st == rpa.RPA_ERR_INVALID
        assert lib.rpa_last_error()
    bad = rpa.rpa.rpa_options()
    lib.rpa_default_options(ctypes.byref(bad))
    bad.n_omega = 0
    st = lib.rpa_setup(ctypes.byref(hd), 4, 4, 4, 0.5, 12, 1, 1, eps, 1, ctypes.byref(bad), None)
    assert st == rpa.RPA_ERR_INVALID and b"n_omega" in lib.rpa_last_error()
    for field, value in (("sq_order", 33), ("stencil_shape", 7), ("z_chunks", -1), ("contractions", 4),
                         ("periodic", 2), ("precondition", 3), ("block_cocg", 17)):
        lib.rpa_default_options(ctypes.byref(bad))
        setattr(bad, field, value)
        st = lib.rpa_setup(ctypes.byref(hd), 4, 4, 4, 0.5, 12, 1, 1, eps, 1, ctypes.byref(bad), None)
        assert st == rpa.RPA_ERR_INVALID and field.encode() in lib.rpa_last_error()


def test_block_cocg_excludes_precondition_and_projection(rpa):
    lib = rpa.library()
    hd = ctypes.c_void_p()
    eps = (ctypes.c_double * 1)(-1.0)
    bad = rpa.rpa.rpa_options()
    for field in ("precondition", "project_solution"):
        lib.rpa_default_options(ctypes.byref(bad))
        bad.block_cocg = 4
        setattr(bad, field, 1)
        st = lib.rpa_setup(ctypes.byref(hd), 4, 4, 4, 0.5, 12, 1, 1, eps, 1, ctypes.byref(bad), None)
        assert st == rpa.RPA_ERR_INVALID and b"block_cocg" in lib.rpa_last_error()


def test_calls_on_null_context_are_rejected(rpa):
    lib = rpa.library()
    assert lib.rpa_coulomb_apply(None, 0.5, 1, 1, 1, None) == rpa.RPA_ERR_INVALID
    assert lib.rpa_apply_nuchi0(None, 0.5, 1, 2, 1, 1, None) == rpa.RPA_ERR_INVALID
    assert lib.rpa_ec(None, 1, 1, None, None, None, None, None) == rpa.RPA_ERR_INVALID
    lib.rpa_destroy(None)
