"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
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
