"""The C-ABI library builds for sm_103a, loads, and exports every function
include/nb.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "nb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for need in ("nb_build_tree", "nb_walk_groups", "nb_forces", "nb_leapfrog_step",
                 "nb_create", "nb_destroy", "nb_direct_sum"):
        assert need in names


def test_library_exports_every_declared_symbol():
    import paper_0909_0541_gb300 as nb
    lib = ctypes.CDLL(nb.library_path())
    missing = [s for s in declared() if not hasattr(lib, s)]
    assert not missing, missing
    assert set(nb.EXPORTED) == set(declared())


def test_error_strings():
    import paper_0909_0541_gb300 as nb
    for code in range(-8, 1):
        assert nb._lib.nb_error_string(code) != b"unknown error"
        assert code == 0 or code in nb.NB_ERR
