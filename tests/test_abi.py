"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/fea.h declares (no GPU needed: nothing is computed here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "fea.h")).read()
    return re.findall(r"^(?:fea_status|const char\*)\s+(fea_\w+)\(", txt, re.M)


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (CUDA runtime first)
    from paper_1802_03433_gb300 import build_lib, fea
    build_lib.build()
    return fea.lib()


def test_header_declares_the_boundary():
    names = set(declared())
    for n in ("fea_mesh_create", "fea_pattern", "fea_assemble", "fea_assemble_backward", "fea_mesh_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    from paper_1802_03433_gb300 import fea
    for code, name in fea.STATUS.items():
        assert lib.fea_status_string(code).decode() == name


def test_null_arguments_rejected_without_gpu(lib):
    import ctypes as C
    from paper_1802_03433_gb300 import fea
    h = C.c_void_p()
    st = lib.fea_mesh_create(None, None, None, 10, None, 0, None, C.byref(h))
    assert st == 1 and b"NULL" in lib.fea_last_error()
    assert lib.fea_mesh_check(None, None) == 1
    assert lib.fea_pattern(None, 1, 1, None, None, None) == 1
    f, c, q = fea.make_form(0, 1), fea.make_coeffs(), fea.make_quadrature(4)
    assert lib.fea_assemble(None, C.byref(f), C.byref(c), C.byref(q), None, None, None) == 1


def test_product_path_has_no_oracle_dependency():
    # the package never imports the oracle (test infrastructure only)
    pkg = os.path.join(ROOT, "paper_1802_03433_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "oracle.cpp" not in src and "liboracle" not in src, f
