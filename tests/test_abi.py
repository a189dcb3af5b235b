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


def test_noalloc_rejects_short_outputs_before_any_call():
    """The wrapper of nb_morton_order_noalloc checks that both outputs hold n
    elements before it reaches the library (host tensors suffice: the check
    raises before any pointer is taken or any kernel launched)."""
    import pytest
    torch = pytest.importorskip("torch")
    import paper_0909_0541_gb300 as nb
    pos = torch.zeros((10, 3), dtype=torch.float64)
    good_k = torch.empty(10, dtype=torch.int64)
    good_p = torch.empty(10, dtype=torch.int32)
    with pytest.raises(ValueError, match="keys_out"):
        nb.morton_order_noalloc(pos, torch.empty(9, dtype=torch.int64), good_p)
    with pytest.raises(ValueError, match="perm_out"):
        nb.morton_order_noalloc(pos, good_k, torch.empty(9, dtype=torch.int32))
    with pytest.raises(ValueError, match="keys_out"):
        nb.morton_order_noalloc(pos, torch.empty((10, 1), dtype=torch.int64), good_p)
