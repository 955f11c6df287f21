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


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the size and field offsets that
    the C compiler gives the header's structs, and the precision constants
    match the header's enum."""
    import subprocess

    import paper_1704_06862_gb300 as sie
    structs = [sie.sie_mlfmm_opts, sie.sie_fill_opts, sie.sie_solve_opts, sie.sie_solve_stats, sie.sie_nn_opts,
               sie.sie_nn_stats]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sie.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{st.__name__} {f} %zu\\n", offsetof({st.__name__}, {f}));')
    for e in ("SIE_PREC_FP64", "SIE_PREC_MIXED", "SIE_PREC_NEAR64"):
        lines.append(f'  printf("enum {e} %d\\n", (int){e});')
    lines += ["  return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(tmp_path / "layout.c"), "-o",
                    str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = ln.split()
        got[(a, b)] = int(v)
    for st in structs:
        assert got[(st.__name__, "size")] == ctypes.sizeof(st), st.__name__
        for f, _ in st._fields_:
            assert got[(st.__name__, f)] == getattr(st, f).offset, (st.__name__, f)
    for e in ("SIE_PREC_FP64", "SIE_PREC_MIXED", "SIE_PREC_NEAR64"):
        assert got[("enum", e)] == getattr(sie, e)
