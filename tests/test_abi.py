"""The C interface without a GPU: the library builds for sm_103a, loads, exports every symbol that
include/qdse.h declares, and rejects bad arguments on the host before touching a device."""
import ctypes
import os
import re

import pytest

from paper_2012_03667_gb300 import build as B
from paper_2012_03667_gb300 import qdse as Q
from paper_2012_03667_gb300 import qdse_mu as QM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return Q.load_library()


def declared_functions(header="qdse.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qdse_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/qdse.h but not exported"
    assert set(names) == set(Q.EXPORTS)
    mu_names = declared_functions("qdse_mu.h")
    for n in mu_names:
        assert hasattr(lib, n), f"{n} declared in include/qdse_mu.h but not exported"
    assert set(mu_names) == set(QM.EXPORTS)
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["qdse.h", "qdse_mu.h"]


def _mu_create(lib, n_ext=2, p_abs=(0.5, 1.0), p4=(0.3, 0.7), q_abs=(0.2, 0.4, 0.9),
               q4=(-1.0, 0.1, 1.2), n_z=4, omega=0.5, precision=Q.QDSE_FP64):
    dp = ctypes.c_double
    arr = lambda xs: (dp * len(xs))(*xs)
    w_q = arr([1.0] * (len(q_abs) * len(q4)))
    z, wz = arr([-0.5, -0.1, 0.2, 0.6][:n_z] + [0.0] * max(0, n_z - 4)), arr([0.5] * n_z)
    p = ctypes.c_void_p()
    st = lib.qdse_mu_grid_create(n_ext, arr(p_abs), arr(p4), len(q_abs), arr(q_abs), len(q4),
                                 arr(q4), w_q, n_z, z, wz, omega, precision, None, ctypes.byref(p))
    return st, p


@pytest.mark.parametrize("kw,msg", [
    (dict(n_ext=0), "n_ext"),
    (dict(p_abs=(0.0, 1.0)), "p_abs"),
    (dict(q_abs=(0.4, 0.2, 0.9)), "increasing"),
    (dict(q4=(0.1, -1.0, 1.2)), "increasing"),
    (dict(q_abs=(0.0, 0.4, 0.9)), "increasing"),
    (dict(p4=(0.3, float("nan"))), "non-finite"),
    (dict(omega=0.0), "omega"),
    (dict(precision=Q.QDSE_MIXED), "precision"),
    (dict(n_z=2000), "n_z"),
])
def test_mu_grid_create_rejects_bad_arguments_on_the_host(lib, kw, msg):
    QM.load_library()
    st, p = _mu_create(lib, **kw)
    assert st == Q.QDSE_ERR_ARG and not p
    assert msg in lib.qdse_mu_last_error().decode()


def test_mu_sweep_rejects_a_null_grid(lib):
    QM.load_library()
    assert lib.qdse_mu_sweep(None, 1, None, 1.0, 0.0, 1.0, 0, None, None, None, None) == Q.QDSE_ERR_ARG
    assert lib.qdse_mu_grid_info(None, None, None) == Q.QDSE_ERR_ARG
    lib.qdse_mu_grid_destroy(None)  # accepted


def test_default_options(lib):
    o = lib.qdse_default_options()
    assert o.precision == Q.QDSE_MIXED and o.vertex == Q.QDSE_VERTEX_BC
    assert o.cf == pytest.approx(4 / 3) and o.tol == 1e-10 and o.alpha == 1.0
    assert o.max_iter == 20000 and o.reuse_kernels == 0 and o.stall_window == 0
    assert o.stop_cycles == 1 and o.shared_kernels == 0


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
                                         ("max_iter", 0), ("tol", float("inf")),
                                         ("stall_window", -1), ("stop_cycles", 2),
                                         ("shared_kernels", 2)])
def test_create_rejects_bad_options(lib, field, value):
    o = lib.qdse_default_options()
    setattr(o, field, value)
    g = Q.qdse_grid(64, 32, 1e-4, 1e4, 0)
    p = ctypes.c_void_p()
    assert lib.qdse_create(ctypes.byref(g), 1, ctypes.byref(o), ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert not p


@pytest.mark.parametrize("field,value,grid_mode,msg", [
    ("vertex", Q.QDSE_VERTEX_RL, 0, "BC vertex"),
    ("precision", Q.QDSE_FP64, 0, "QDSE_MIXED"),
    ("precision", Q.QDSE_FP64_PRE, 0, "QDSE_MIXED"),
    (None, None, 1, "COLLOCATED"),
])
def test_shared_kernels_needs_bc_mixed_and_one_collocated_grid(lib, field, value, grid_mode, msg):
    """The tensor-core sweep of a shared-kernel batch covers the BC vertex on one collocated grid
    with FP32 Picard sweeps; anything else is refused before any device work."""
    o = lib.qdse_default_options()
    o.shared_kernels = 1
    if field:
        setattr(o, field, value)
    g = Q.qdse_grid(64, 32, 1e-4, 1e4, grid_mode)
    p = ctypes.c_void_p()
    assert lib.qdse_create(ctypes.byref(g), 4, ctypes.byref(o), ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert not p and msg in lib.qdse_last_error(None).decode()
    if field is None:
        return
    o.vertex, o.precision = Q.QDSE_VERTEX_BC, Q.QDSE_MIXED
    two = (Q.qdse_grid * 2)(Q.qdse_grid(64, 32, 1e-4, 1e4, 0), Q.qdse_grid(64, 32, 1e-4, 1e4, 0))
    assert lib.qdse_create_ragged(two, 2, ctypes.byref(o), ctypes.byref(p)) == Q.QDSE_ERR_ARG
    assert "qdse_create" in lib.qdse_last_error(None).decode()


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
    assert lib.qdse_autotune(None, None, None, None, 5, None, None) == Q.QDSE_ERR_ARG
    lib.qdse_destroy(None)  # accepted


@pytest.mark.parametrize("kw,msg", [
    (dict(p_axis=(0.5, 0.2)), "axes"),
    (dict(p_axis=(0.0, 0.2)), "axes"),
    (dict(p4_axis=(-0.1, 0.3)), "axes"),
    (dict(n_pr=0), "axis"),
])
def test_mu_product_grid_and_solve_reject_bad_arguments_on_the_host(lib, kw, msg):
    QM.load_library()
    dp = ctypes.c_double
    arr = lambda xs: (dp * len(xs))(*xs)
    a = dict(n_pr=2, p_axis=(0.2, 0.5), p4_axis=(0.1, 0.4))
    a.update(kw)
    q_abs, q4 = arr([0.3, 0.6]), arr([-0.2, 0.2])
    p = ctypes.c_void_p()
    st = lib.qdse_mu_grid_create_product(a["n_pr"], arr(a["p_axis"]), len(a["p4_axis"]),
                                         arr(a["p4_axis"]), 2, q_abs, 2, q4, arr([1.0] * 4), 2,
                                         arr([-0.5, 0.5]), arr([1.0, 1.0]), 0.5, Q.QDSE_FP64,
                                         None, ctypes.byref(p))
    assert st == Q.QDSE_ERR_ARG and not p
    assert msg in lib.qdse_mu_last_error().decode()
    assert lib.qdse_mu_solve(None, None, 1, None, 1.0, 0.0, 1.0, 0, 1.0, 1e-10, 1e-5, 10, None,
                             None, None, None) == Q.QDSE_ERR_ARG


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_public_headers_compile_as_plain_c_and_cxx(tmp_path, lang, std):
    """include/*.h is a C ABI: both headers compile on their own and together as C99 (no C++
    types, no torch types) and as C++, with every warning an error."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("use.c" if lang == "c" else "use.cpp")
    src.write_text('#include "qdse.h"\n#include "qdse_mu.h"\n#include "qdse.h"\n'
                   "int main(void) { qdse_mu_grid* g = 0; qdse_ctx* c = 0; (void)g; (void)c;\n"
                   "  return QDSE_OK + QDSE_VERTEX_BC + QDSE_FP32; }\n")
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
