"""The C ABI's argument checks on the host, without a GPU: every entry point that takes a handle
returns MFNS_ERR_ARG for a null one (null outputs and zero sizes alongside), records a message for
mfns_last_error, and the destroy calls accept null.  None of these calls reaches the device."""
import ctypes as C

import pytest

from paper_2603_29621_gb300 import _lib

NULL_OK = {"mfns_ctx_destroy", "mfns_mesh_destroy", "mfns_problem_destroy", "mfns_spacetime_destroy"}
NOT_HANDLE = {"mfns_last_error", "mfns_spacetime_temporal"}


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    return C.CDLL(_lib.LIB_PATH)


def _call_with_nulls(lib, name):
    res, args = _lib._SIGS[name]
    f = getattr(lib, name)
    f.restype, f.argtypes = res, args
    vals = [0 if a in (C.c_int, C.c_int64, C.c_size_t, C.c_uint32) else 0.0 if a is C.c_double else None
            for a in args]
    return f(*vals)


@pytest.mark.parametrize("name", sorted(set(_lib._SIGS) - NULL_OK - NOT_HANDLE))
def test_null_handle_is_an_argument_error(lib, name):
    assert _call_with_nulls(lib, name) == _lib.ERR_ARG
    last = lib.mfns_last_error
    last.restype = C.c_char_p
    assert last()  # a message explains the failure


@pytest.mark.parametrize("name", sorted(NULL_OK))
def test_destroying_null_is_a_no_op(lib, name):
    assert _call_with_nulls(lib, name) == _lib.OK


def test_temporal_tables_check_the_order(lib):
    f = lib.mfns_spacetime_temporal
    res, args = _lib._SIGS["mfns_spacetime_temporal"]
    f.restype, f.argtypes = res, args
    nulls = [None] * (len(args) - 1)
    assert f(-1, *nulls) == _lib.ERR_ARG
    assert f(8, *nulls) == _lib.ERR_ARG
    assert f(7, *nulls) == _lib.OK          # every output pointer may be null
