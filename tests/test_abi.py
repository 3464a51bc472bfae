"""The C-ABI library builds, loads and exports every function include/bem.h
declares; argument errors come back as status codes (no GPU needed)."""
import ctypes

import pytest

from paper_2003_12663_gb300 import bem, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return bem.lib()


def test_every_header_symbol_is_exported(L):
    names = bem.header_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(bem._SIGS), set(names) ^ set(bem._SIGS)


def test_default_params(L):
    p = bem.default_params()
    assert p.eta == 4.0 and p.far_order == 3 and p.gmres_restart == 100


def test_argument_errors_without_device(L):
    h = ctypes.c_void_p()
    assert L.bem_create(None, None, None, None) == -1
    assert L.bem_create(ctypes.byref(h), None, None, None) == -1
    assert b"NULL" in L.bem_last_error(None)
    m = bem.bem_mesh()
    m.nv, m.np = 3, 1
    assert L.bem_create(ctypes.byref(h), ctypes.byref(m), None, None) == -1
    assert not h.value
    # calls on a NULL context are argument errors
    assert L.bem_matvec(None, 0, 1, None, None) == -1
    assert L.bem_solve(None, 0, 1, None, None, 1e-8, None, None) == -1
    assert L.bem_eval_field(None, 0, None, 0, None, None, None) == -1
    assert L.bem_destroy(None) == 0


def test_bad_mesh_rejected_before_device(L):
    import numpy as np
    X = np.zeros((3, 3))
    tri = np.array([[0, 1, 5]], np.int32)
    reg = np.zeros(1, np.int32)
    regs = (bem.bem_region * 1)()
    m = bem.bem_mesh(3, 1, X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                     reg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1, regs)
    h = ctypes.c_void_p()
    assert L.bem_create(ctypes.byref(h), ctypes.byref(m), None, None) == -1
    assert b"out of range" in L.bem_last_error(None)
    p = bem.default_params(eta=0.5)
    tri[0, 2] = 2
    assert L.bem_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(p), None) == -1
    assert b"eta" in L.bem_last_error(None)
