"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/grte.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "grte.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grte(?:2d)?_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1811_05579_gb300 import build
    if not os.path.exists(build.LIB) or any(
            os.path.getmtime(s) > os.path.getmtime(build.LIB) for s in build.SOURCES):
        build.build_library()
    return build.LIB


def test_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1811_05579_gb300 import grte
    assert sorted(grte.EXPORTED) == _declared()


def test_null_handle_calls_are_rejected(libpath):
    from paper_1811_05579_gb300 import grte
    L = grte.load_library(libpath)
    assert L.grte_step(None, 1) == 1          # EINVAL, no CUDA call made
    assert L.grte_sync(None) == 1
    L.grte_destroy(None)                       # no-op
    assert L.grte2d_step(None, 1) == 1
    L.grte2d_destroy(None)
