"""The C-ABI library builds, loads without a GPU and exports every entry point of include/mfns.h."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mfns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mfns_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mfns_ctx_create", "mfns_mesh_uniform", "mfns_mesh_refine_ball", "mfns_problem_create",
                     "mfns_vmult", "mfns_smooth", "mfns_vcycle", "mfns_solve", "mfns_apply_constraints",
                     "mfns_restrict", "mfns_prolongate_add", "mfns_diagonal"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    from paper_2603_29621_gb300 import _lib

    g.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding's signature table covers the header
    assert set(declared_functions()) <= set(_lib.EXPORTED)
