"""The C-ABI library builds for sm_103a, loads, exports every symbol that
include/adm.h declares, and rejects bad arguments / meshes on the host
(no GPU needed: these checks run before any CUDA call)."""
import ctypes as C

import numpy as np
import pytest

import __graft_entry__
import paper_2509_00406_gb300 as adm


@pytest.fixture(scope="module")
def L():
    __graft_entry__.build()
    return adm.lib()


def test_exports_every_declared_symbol(L):
    names = adm.declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_strerror(L):
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert len(adm.strerror(s)) > 0


def _create(L, V, F, var_dim=3):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    h = C.c_void_p()
    s = L.adm_create(V.ctypes.data_as(C.c_void_p), V.shape[0], F.ctypes.data_as(C.c_void_p), F.shape[0],
                     var_dim, C.byref(h))
    return s, h


def test_create_rejects_bad_input(L):
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.float64)
    F = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    assert L.adm_create(None, 4, None, 2, 3, None) == -1
    assert _create(L, V, F, var_dim=4)[0] == -1                              # var_dim
    assert _create(L, V, np.array([[0, 1, 7]]))[0] == -2                     # index out of range
    assert _create(L, V, np.array([[0, 1, 1]]))[0] == -2                     # repeated vertex
    Vd = V.copy()
    Vd[2] = [2.0, 0.0, 0.0]                                                   # collinear rest triangle
    assert _create(L, Vd, np.array([[0, 1, 2]]))[0] == -2
    Vn = V.copy()
    Vn[0, 0] = np.nan
    assert _create(L, Vn, F)[0] == -2
    # batch: a face indexing another mesh's vertices is a mesh error
    vo = np.array([0, 3, 4], dtype=np.int64)
    fo = np.array([0, 1, 2], dtype=np.int64)
    h = C.c_void_p()
    s = L.adm_create_batch(V.ctypes.data_as(C.c_void_p), vo.ctypes.data_as(C.c_void_p),
                           F.ctypes.data_as(C.c_void_p), fo.ctypes.data_as(C.c_void_p), 2, 3, C.byref(h))
    assert s == -2


def test_null_handle_calls(L):
    assert L.adm_get_status(None) == -1
    assert L.adm_eval(None, 1, 0, None, None, None, None, None) == -1
    assert L.adm_set_params(None, 2, None, 0) == -1
    L.adm_destroy(None)
