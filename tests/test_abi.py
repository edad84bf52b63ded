"""The C-ABI library loads and exports every entry point include/cflr.h
declares (no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "cflr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cflr_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for need in ("cflr_load_grammar", "cflr_load_graph", "cflr_solve", "cflr_get_pairs",
                 "cflr_solve_batch", "cflr_create", "cflr_destroy", "cflr_last_error"):
        assert need in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2401_11029_gb300 import build, cflr
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    assert sorted(cflr.EXPORTS) == declared_entry_points()


def test_checked_library_builds_and_exports_every_symbol():
    """The bounds-checked build (CFLR_CHECKED) is the same library."""
    from paper_2401_11029_gb300 import build
    build.build()
    lib = ctypes.CDLL(build.LIB_CHECKED)
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_names_match_the_c_abi():
    import paper_2401_11029_gb300 as pkg
    from paper_2401_11029_gb300 import cflr
    for name in declared_entry_points():
        assert hasattr(cflr, name), name


def test_oracle_is_not_imported_by_the_product():
    import subprocess
    import sys
    code = ("import sys; import paper_2401_11029_gb300 as p; "
            "from paper_2401_11029_gb300 import cflr, gen, build; "
            "assert 'oracle' not in sys.modules, 'product imported the oracle'")
    subprocess.check_call([sys.executable, "-c", code], cwd=ROOT)
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2401_11029_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
