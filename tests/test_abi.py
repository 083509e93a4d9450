"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (no GPU calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\S[^\n;(]*?\b(bchdav_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("bchdav_create", "bchdav_destroy", "bchdav_build_laplacian", "bchdav_solve",
                     "bchdav_filter", "bchdav_orthonormalize", "bchdav_eigh", "bchdav_spmm",
                     "bchdav_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2212_04443_gb300 as P
    L = P.lib()
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing
    assert sorted(P.EXPORTED_SYMBOLS) == declared_symbols()


def test_status_strings():
    import paper_2212_04443_gb300 as P
    L = P.lib()
    assert L.bchdav_status_string(0) == b"ok"
    assert b"CSR" in L.bchdav_status_string(-2)
    assert L.bchdav_status_string(123) == b"unknown status"


def test_package_has_no_oracle_dependency():
    pkg = os.path.join(ROOT, "paper_2212_04443_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "oracle/" not in txt, f
