"""The C-ABI library loads (symbol table) and exports every entry point include/sgtn.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sgtn.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int(?:32|64)_t|int|void|const char\s*\*)\s*(sgtn_\w+)\s*\(", txt, re.M)))


def test_library_exports_all_declared_symbols():
    from paper_2411_16431_b300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (sgtn_\w+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    # dlopen works on a machine without a GPU too (no compute call is made)
    L = ctypes.CDLL(lib)
    for s in _declared():
        assert hasattr(L, s)
