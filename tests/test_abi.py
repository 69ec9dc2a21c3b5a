"""The C interface without a GPU: the library builds for sm_103a, loads, exports every symbol that
include/qdse.h declares, and rejects bad arguments on the host before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2012_03667_gb300 import build as B
from paper_2012_03667_gb300 import qdse as Q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return Q.load_library()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qdse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qdse_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/qdse.h but not exported"
    assert set(names) == set(Q.EXPORTS)


def test_default_options(lib):
    o = lib.qdse_default_options()
    assert o.precision == Q.QDSE_MIXED and o.vertex == Q.QDSE_VERTEX_BC
    assert o.cf == pytest.approx(4 / 3) and o.tol == 1e-10 and o.alpha == 1.0
    assert o.max_iter == 20000 and o.reuse_kernels == 0


@pytest.mark.parametrize("grid,msg", [
    (Q.qdse_grid(2, 32, 1e-4, 1e4, 0), "n_p"),
    (Q.qdse_grid(2000, 32, 1e-4, 1e4, 0), "n_p"),
    (Q.qdse_grid(64, 0, 1e-4, 1e4, 0), "n_theta"),
    (Q.qdse_grid(64, 32, -1.0, 1e4, 0), "s_min"),
    (Q.qdse_grid(64, 32, 1e4, 1e-4, 0), "s_min"),
    (Q.qdse_grid(64, 32, float("nan"), 1e4, 0), "s_min"),
    (Q.qdse_grid(64, 32, 1e-4, 1e4, 7), "grid_mode"),
])
def test_create_rejects_bad_grids(lib, grid, msg):
    o = lib.qdse_default_options()
    p = ctypes.c_void_p()
    st = lib.qdse_create(ctypes.byref(grid), 1, ctypes.byref(o), ctypes.byref(p))
    assert st == Q.QDSE_ERR_ARG and not p
    assert msg in lib.qdse_last_error(None).decode()


@pytest.mark.parametrize("field,value", [("precision", 9), ("vertex", 3), ("cf", 0.0),
                                         ("tol", -1.0), ("alpha", 0.0), ("alpha", 1.5),
                                         ("max_iter", 0), ("tol", float("inf"))])
def test_create_rejects_bad_options(lib, field, value):
    o = lib.qdse_default_options()
    setattr(o, field, value)
    g = Q.qdse_grid(64, 32, 1e-4, 1e4, 0)
    p = ctypes.c_void_p()
    assert lib.qdse_create(ctypes.byref(g), 1, ctypes.byref(o), ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert not p


def test_create_rejects_null_and_empty(lib):
    o = lib.qdse_default_options()
    g = Q.qdse_grid(64, 32, 1e-4, 1e4, 0)
    p = ctypes.c_void_p()
    assert lib.qdse_create(None, 1, ctypes.byref(o), ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert lib.qdse_create(ctypes.byref(g), 0, ctypes.byref(o), ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert lib.qdse_create(ctypes.byref(g), 1, None, ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert lib.qdse_create(ctypes.byref(g), 1, ctypes.byref(o), None) == Q.QDSE_ERR_ARG
    bad = (Q.qdse_grid * 2)(Q.qdse_grid(64, 32, 1e-4, 1e4, 0), Q.qdse_grid(64, 32, 1e-4, 1e4, 5))
    assert lib.qdse_create_ragged(bad, 2, ctypes.byref(o), ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert "instance 1" in lib.qdse_last_error(None).decode()


def test_null_context_is_rejected(lib):
    assert lib.qdse_solve(None, None, None, None, None, None) == Q.QDSE_ERR_ARG
    assert lib.qdse_sizes(None, None, None) == Q.QDSE_ERR_ARG
    lib.qdse_destroy(None)  # accepted
