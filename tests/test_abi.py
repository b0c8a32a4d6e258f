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
