"""The C-ABI library builds, loads and exports every symbol include/heom.h declares.

No compute call is made here (this file runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "heom.h")
LIB = os.path.join(ROOT, "paper_2306_07522_gb300", "libheom.so")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(heom_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("heom_build_hierarchy", "heom_apply", "heom_evolve", "heom_steady",
                     "heom_spectrum", "heom_destroy", "heom_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_exactly_the_declared_symbols(lib):
    import paper_2306_07522_gb300 as heom
    assert sorted(heom.EXPORTED) == _declared()


def test_binding_has_no_cpu_fallback():
    """The package must not import the oracle or any CPU implementation of the path."""
    pkg = os.path.join(ROOT, "paper_2306_07522_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src, f
                assert "scipy" not in src, f
