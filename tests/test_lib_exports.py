"""CPU checks of the boundary: the native library loads and exports every
function include/tmat.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tmat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\s*\*)\s*(tmat_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["tmat_build", "tmat_solve", "tmat_adjoint", "tmat_field", "tmat_farfield", "tmat_neighbors",
              "tmat_subregions", "tmat_apply", "tmat_translation", "tmat_incident_planewave"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2107_09879_b300 import build
    lib_path = build.build(verbose=False)
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2107_09879_b300 import _lib
    assert set(_declared()) <= set(_lib.EXPORTED)
