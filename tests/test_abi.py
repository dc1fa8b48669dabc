"""The C-ABI library builds, loads and exports every function include/trw.h
declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import paper_2107_11983_gb300 as trw
from paper_2107_11983_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "trw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(trw_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_functions():
    assert sorted(trw._SIGS) == declared_functions()


def test_binding_loads_without_gpu():
    lib = trw.load_library()
    assert lib.trw_last_error() is not None
