"""CPU checks of the C ABI: the library builds, loads, and exports every
function ``include/sie.h`` declares (no compute call without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[\w\s\*]+?)\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "sizeof", "return")))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1704_06862_gb300 import build
    return build.build()


def test_header_declares_the_abi():
    names = _declared()
    for required in ("sie_build_mesh", "sie_fill_nearfield", "mlfmm_setup", "mlfmm_matvec", "ilu_apply",
                     "gmres_solve", "rcs_farfield"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_loads_and_names_match(lib_path):
    import paper_1704_06862_gb300 as sie
    sie.load_library(lib_path)
    assert sorted(sie.EXPORTED) == _declared()
    for name in sie.EXPORTED:
        assert callable(getattr(sie, name))


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    import paper_1704_06862_gb300 as sie
    mod = importlib.reload(sie)
    with pytest.raises(RuntimeError):
        mod.load_library(str(tmp_path / "missing.so"))
    importlib.reload(sie)
