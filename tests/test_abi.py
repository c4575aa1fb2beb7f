"""The C ABI library builds, loads and exports every function that include/sfcoct.h
declares; the oracle library builds too.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

import oracle
import paper_2603_06771_gb300 as sfc
from paper_2603_06771_gb300 import binding
from conftest import ROOT


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sfcoct.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"^\s*typedef[^;]*;", "", text, flags=re.M | re.S)  # function-pointer types are not entry points
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("octree_build", "radius_search", "knn", "octree_free", "sfc_csr_free", "sfc_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = sfc.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    assert set(declared_functions()) <= set(binding._SIGNATURES)


def test_status_strings():
    lib = binding.lib()
    for code in range(9):
        assert lib.sfc_status_string(code)
    assert lib.sfc_launch_count() >= 0


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB", os.path.join(ROOT, "no", "such", "libsfcoct.so"))
    with pytest.raises(RuntimeError):
        binding.lib()


def test_oracle_library_builds():
    assert os.path.exists(oracle.build())
