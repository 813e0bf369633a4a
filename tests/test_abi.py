"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol; the
header is plain C and C++, and the binding's struct layout and argument counts match it."""
import os
import re

import pytest

from paper_2011_01400_gb300 import build as B
from paper_2011_01400_gb300 import gw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    return sorted(set(re.findall(r"^\s*(?:gw_status|const char\*|size_t)\s+(gw_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("gw_plan_create", "gw_chi0", "gw_screen", "gw_sigma", "gw_qp", "gw_plan_destroy", "gw_last_error"):
        assert n in names
    assert set(names) == set(gw.EXPORTS)


@pytest.mark.skipif(B.shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no CUDA toolkit")
def test_library_builds_loads_and_exports():
    B.build()
    lib = gw.load()
    for n in declared_symbols():
        assert hasattr(lib, n), n
    assert lib.gw_last_error() is not None
    assert lib.gw_problem_bytes() == gw.ctypes.sizeof(gw.gw_problem)


def test_struct_layout_matches_header():
    # offsets of the C struct as laid out on LP64: pointers 8-aligned, doubles 8-aligned
    p = gw.gw_problem
    assert p.nk.offset == 0
    assert p.basis_atom.offset == 32
    assert p.eps.offset % 8 == 0 and p.qhat.offset % 8 == 0
    assert p.prec.offset + 4 <= gw.ctypes.sizeof(p)
    assert p.time_reversal.offset == p.prec.offset + 4
    assert p.freq.offset == p.k_offset.offset + 24 and p.freq_w.offset == p.freq.offset + 8
    assert gw.ctypes.sizeof(p) == p.freq_w.offset + 8


def test_null_arguments_are_rejected_without_gpu():
    B.build()
    lib = gw.load()
    h = gw.ctypes.c_void_p()
    assert lib.gw_plan_create(None, 1, None, gw.ctypes.byref(h)) == gw.GW_ERR_ARG
    assert b"NULL" in lib.gw_last_error()
    assert lib.gw_chi0(None, 0, 0, None) == gw.GW_ERR_ARG
    assert lib.gw_plan_destroy(None) == gw.GW_OK


@pytest.mark.skipif(B.shutil.which("gcc") is None, reason="no C compiler")
def test_header_is_plain_c_and_cxx(tmp_path):
    """include/gw.h compiles on its own as C99 and as C++11 (pedantic, warnings as errors), and a C
    caller's sizeof(gw_problem) equals the library's."""
    import subprocess
    inc = os.path.join(ROOT, "include")
    src = tmp_path / "caller.c"
    src.write_text('#include "gw.h"\n#include <stdio.h>\n'
                   'int main(void) { printf("%zu %zu\\n", sizeof(gw_problem), gw_problem_bytes()); return 0; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, "-c", str(src),
                    "-o", str(tmp_path / "caller.o")], check=True)
    cxx = tmp_path / "caller.cpp"
    cxx.write_text('#include "gw.h"\nint main() { return sizeof(gw_problem) > 0 ? 0 : 1; }\n')
    if B.shutil.which("g++"):
        subprocess.run(["g++", "-std=c++11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, "-c", str(cxx),
                        "-o", str(tmp_path / "caller_cxx.o")], check=True)
    B.build()
    lib_dir = os.path.dirname(gw.LIB_PATH)
    exe = tmp_path / "caller"
    subprocess.run(["gcc", str(tmp_path / "caller.o"), "-L", lib_dir, "-lgw", "-Wl,-rpath," + lib_dir, "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out[0] == out[1]


def test_binding_argument_counts_match_the_header():
    """Every declared entry point has as many ctypes argument types in the binding as the header
    declares parameters (a dropped or extra argument would shift every pointer after it)."""
    src = open(os.path.join(ROOT, "include", "gw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    decls = re.findall(r"(?:gw_status|const char\*|size_t)\s+(gw_\w+)\s*\(([^)]*)\)\s*;", src)
    assert len(decls) == len(gw.EXPORTS)
    B.build()
    lib = gw.load()
    for name, args in decls:
        a = args.strip()
        n = 0 if a in ("", "void") else a.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, name
