"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/claire.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2008_12820_gb300 import build as B
from paper_2008_12820_gb300 import claire

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "claire.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(claire_[A-Za-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    # the Python binding covers the same entry points
    assert set(claire.EXPORTED) == set(names)


def test_binding_refuses_without_library(tmp_path):
    import pytest
    with pytest.raises(RuntimeError):
        claire._lib = None
        claire.load(str(tmp_path / "missing.so"))
    claire._lib = None
