"""The C-ABI library builds, loads and exports every entry point that
include/cardiac_bddc.h declares (no compute calls: runs without a GPU)."""
import os
import re

import pytest

import paper_2208_06191_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"CBDDC_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)
    return names


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fem_assemble_tangent", "bddc_setup", "bddc_apply", "newton_gmres_solve"):
        assert required in names
    assert sorted(names) == sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    assert sorted(names) == sorted(pkg.EXPORTED_SYMBOLS)


def test_error_string_is_available_without_a_gpu(lib):
    assert isinstance(lib.cbddc_last_error(), bytes)


# ctypes mirror -> C struct of the header
_STRUCTS = {
    "_Desc": "fem_problem_desc", "_ProblemInfo": "fem_problem_info", "_Tangent": "fem_tangent",
    "_BddcOptions": "bddc_options", "_BddcInfo": "bddc_info", "_GmresOptions": "gmres_options",
    "_GmresReport": "gmres_report", "_SolveOptions": "solve_options", "_Record": "newton_record",
    "_Report": "solve_report",
}
_ENUMS = {
    "OK": "CBDDC_OK", "EINVAL": "CBDDC_EINVAL", "ECUDA": "CBDDC_ECUDA", "EPIVOT": "CBDDC_EPIVOT",
    "EINVERTED": "CBDDC_EINVERTED", "ENOCONV": "CBDDC_ENOCONV", "ETIMEOUT": "CBDDC_ETIMEOUT",
    "ENOMEM": "CBDDC_ENOMEM", "HEX_Q1": "CBDDC_HEX_Q1", "HEX_Q2": "CBDDC_HEX_Q2",
    "TET_P1": "CBDDC_TET_P1", "TET_P2": "CBDDC_TET_P2", "FP64": "CBDDC_FP64", "FP32": "CBDDC_FP32",
    "PRIMAL_V": "CBDDC_PRIMAL_V", "PRIMAL_E": "CBDDC_PRIMAL_E", "PRIMAL_F": "CBDDC_PRIMAL_F",
    "PRIMAL_R": "CBDDC_PRIMAL_R", "SCALING_COUNTING": "CBDDC_SCALING_COUNTING",
    "SCALING_DELUXE": "CBDDC_SCALING_DELUXE", "COARSE_GALERKIN": "CBDDC_COARSE_GALERKIN",
    "COARSE_PETROV": "CBDDC_COARSE_PETROV", "FIBER_SLAB_HELIX": "CBDDC_FIBER_SLAB_HELIX",
    "FIBER_NODAL": "CBDDC_FIBER_NODAL", "TIMER_SWEEP_GEMM": "CBDDC_TIMER_SWEEP_GEMM",
    "TIMER_APPLY": "CBDDC_TIMER_APPLY", "TIMER_SETUP": "CBDDC_TIMER_SETUP",
    "TIMER_LEVEL2_SETUP": "CBDDC_TIMER_LEVEL2_SETUP", "TIMER_LEVEL2_APPLY": "CBDDC_TIMER_LEVEL2_APPLY",
    "TIMER_COARSE_SETUP": "CBDDC_TIMER_COARSE_SETUP", "TIMER_COARSE_APPLY": "CBDDC_TIMER_COARSE_APPLY",
    "TIMER_SETUP_GEMM_F64": "CBDDC_TIMER_SETUP_GEMM_F64",
}


def test_ctypes_mirrors_match_the_header(tmp_path):
    # compile a host program against the header (plain C) and compare every
    # struct's size and field offsets, and the enum values, with the binding
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cardiac_bddc.h"', "int main(void) {"]
    for py, c in _STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (py, c))
        for field, _ in getattr(pkg, py)._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (py, field, c, field))
    for py, c in _ENUMS.items():
        lines.append('printf("enum %s %%d\\n", (int)%s);' % (py, c))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for py in _STRUCTS:
        st = getattr(pkg, py)
        assert got[(py, "size")] == ctypes.sizeof(st), py
        for field, _ in st._fields_:
            assert got[(py, field)] == getattr(st, field).offset, (py, field)
    for py, c in _ENUMS.items():
        assert got[("enum", py)] == getattr(pkg, py), c
