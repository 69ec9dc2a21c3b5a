"""FP64 CPU oracle for the vacuum quark gap equation with the Ball-Chiu vertex.

TEST INFRASTRUCTURE ONLY.  ``qdse_oracle.cpp`` (plain C++ loops, FP64) is the independent checker
of the GPU solver; this module compiles it with the host ``g++`` and wraps its C interface with
``ctypes`` and numpy.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It imports nothing from the GPU package.

Every function follows the paper (arXiv:2012.03667) section it names; the readings taken where the
paper is garbled (R1-R10) are listed in the header of ``qdse_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qdse_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (host g++, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        grid_args = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                     ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.c_double]
        lib.oracle_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
        lib.oracle_angular_grid.argtypes = [ctypes.c_int, _dp, _dp, _dp]
        lib.oracle_angular_grid.restype = None
        lib.oracle_radial_grid.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, _dp, _dp, _dp, _ip]
        lib.oracle_values_at_q.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, _dp, _dp]
        lib.oracle_point_integrand.argtypes = [ctypes.c_double] * 9 + [ctypes.c_int, _dp, _dp]
        lib.oracle_point_integrand.restype = None
        lib.oracle_diag_quotient.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int]
        lib.oracle_diag_quotient.restype = ctypes.c_double
        lib.oracle_sweep.argtypes = grid_args + [_dp, _dp, _dp, _dp, ctypes.c_int]
        lib.oracle_solve.argtypes = grid_args + [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                 _dp, _dp, _ip, _dp, ctypes.c_int]
        lib.oracle_jacobian.argtypes = grid_args + [_dp, _dp, _dp, ctypes.c_int]
        lib.oracle_param_jacobian.argtypes = grid_args + [_dp, _dp, _dp]
        lib.oracle_adjoint.argtypes = grid_args + [_dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        lib.oracle_condensate.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, _dp, _dp]
        lib.oracle_condensate.restype = ctypes.c_double
        lib.oracle_num_threads_available.argtypes = []
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype=_dp):
    return a.ctypes.data_as(ctype)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


COLLOCATED, STAGGERED = 0, 1
# The staggered grid with the paper's traditional interpolation (Table 1, algorithms 1 and 3):
# the bracket of each internal node is searched for at every integrand evaluation.  Same values
# as STAGGERED, more work; for timing the paper's comparison only.
STAGGERED_TRADITIONAL = 2
BC, RL = 0, 1
STATUS = {0: "converged", 1: "bad argument", 4: "not converged", 5: "non-finite"}


@dataclass
class Problem:
    """One gap-equation instance: grid (Sec. IV parameters N, M), interaction (Eq. IRGsQC),
    current mass (Eq. gendse) and vertex choice."""
    n: int = 64
    n_theta: int = 32
    s_min: float = 1e-4
    s_max: float = 1e4
    grid_mode: int = COLLOCATED
    vertex: int = BC
    cf: float = 4.0 / 3.0
    D: float = 0.93
    omega: float = 0.5
    m: float = 0.005

    def _args(self):
        return (self.n, self.n_theta, self.s_min, self.s_max, self.grid_mode, self.vertex,
                self.cf, self.D, self.omega, self.m)


def gauss_legendre(n: int):
    """Gauss-Legendre nodes (ascending) and weights on [-1, 1] (Sec. II discretisation)."""
    lib = _load()
    t = np.zeros(n); v = np.zeros(n)
    if lib.oracle_gauss_legendre(n, _ptr(t), _ptr(v)):
        raise ValueError("bad n")
    return t, v


def angular_grid(m: int):
    """Gauss-Chebyshev (2nd kind) nodes z_k, 1 - z_k and weights w_k (reading R10)."""
    lib = _load()
    z = np.zeros(m); y = np.zeros(m); w = np.zeros(m)
    lib.oracle_angular_grid(m, _ptr(z), _ptr(y), _ptr(w))
    return z, y, w


def radial_grid(n: int, s_min: float = 1e-4, s_max: float = 1e4, grid_mode: int = COLLOCATED):
    """External grid s_p, internal grid s_q, weights W (int ds s f = sum W f) and, for the
    staggered grid, the bracket of each q_j found by the traditional search (Eq. chazhiresult0)."""
    lib = _load()
    sp = np.zeros(n); sq = np.zeros(n); W = np.zeros(n); br = np.zeros(n, dtype=np.int32)
    if lib.oracle_radial_grid(n, s_min, s_max, grid_mode, _ptr(sp), _ptr(sq), _ptr(W),
                              _ptr(br, _ip)):
        raise ValueError("bad grid")
    return sp, sq, W, br


def values_at_q(F, s_min: float = 1e-4, s_max: float = 1e4, grid_mode: int = COLLOCATED):
    """F at the internal nodes: on-grid, or the modified interpolation (Eq. chazhiresult)."""
    lib = _load()
    F = _f64(F)
    Fq = np.zeros(len(F))
    if lib.oracle_values_at_q(len(F), s_min, s_max, grid_mode, _ptr(F), _ptr(Fq)):
        raise ValueError("bad grid")
    return Fq


def point_integrand(P, Q, z, Ap, Bp, Aq, Bq, DA, DB, vertex=BC):
    """Reduced I_A, I_B of Eqs. dsesys/dsesys2 at one (P, Q, z), without interaction/measure."""
    lib = _load()
    ia = ctypes.c_double(); ib = ctypes.c_double()
    lib.oracle_point_integrand(P, Q, z, Ap, Bp, Aq, Bq, DA, DB, vertex, ctypes.byref(ia),
                               ctypes.byref(ib))
    return ia.value, ib.value


def diag_quotient(s, F, i: int) -> float:
    """dF/ds at node i from the 3-point Lagrange stencil in ln s (reading R8)."""
    lib = _load()
    s = _f64(s); F = _f64(F)
    return lib.oracle_diag_quotient(_ptr(s), len(s), _ptr(F), i)


def sweep(pr: Problem, A, B, nthreads: int = 1):
    """One Jacobi successive-approximation sweep x -> F(x) (Eq. jifen12, reading R6)."""
    lib = _load()
    A = _f64(A); B = _f64(B)
    Ao = np.zeros(pr.n); Bo = np.zeros(pr.n)
    if lib.oracle_sweep(*pr._args(), _ptr(A), _ptr(B), _ptr(Ao), _ptr(Bo), nthreads):
        raise ValueError("bad problem")
    return Ao, Bo


def solve(pr: Problem, A0=1.0, B0=0.3, tol: float = 1e-10, alpha: float = 1.0,
          max_iter: int = 2000, nthreads: int = 1):
    """Successive approximation from (A0, B0) to the R7 tolerance (Eqs. jifen14-jifenab2).
    Returns (A, B, iterations, last max relative change, status)."""
    lib = _load()
    A = _f64(np.broadcast_to(A0, (pr.n,))).copy(); B = _f64(np.broadcast_to(B0, (pr.n,))).copy()
    it = ctypes.c_int(); ch = ctypes.c_double()
    st = lib.oracle_solve(*pr._args(), tol, alpha, max_iter, _ptr(A), _ptr(B), ctypes.byref(it),
                          ctypes.byref(ch), nthreads)
    return A, B, it.value, ch.value, st


def jacobian(pr: Problem, A, B, nthreads: int = 1) -> np.ndarray:
    """dF/dx at x = (A, B) by the complex step, 2n x 2n, ordered (A..., B...)."""
    lib = _load()
    A = _f64(A); B = _f64(B)
    J = np.zeros((2 * pr.n, 2 * pr.n))
    if lib.oracle_jacobian(*pr._args(), _ptr(A), _ptr(B), _ptr(J), nthreads):
        raise ValueError("bad problem")
    return J


def param_jacobian(pr: Problem, A, B) -> np.ndarray:
    """dF/d(m, D, omega) at fixed x by the complex step, 3 x 2n."""
    lib = _load()
    A = _f64(A); B = _f64(B)
    dF = np.zeros((3, 2 * pr.n))
    if lib.oracle_param_jacobian(*pr._args(), _ptr(A), _ptr(B), _ptr(dF)):
        raise ValueError("bad problem")
    return dF


def adjoint(pr: Problem, A, B, gA, gB, nthreads: int = 1):
    """Implicit-function adjoint at a fixed point: (I - J^T) lambda = g, then
    dL/d(m, D, omega, mu) = lambda^T dF/dtheta (mu does not enter the vacuum equation: 0).
    Returns (gparams[4], lambda[2n])."""
    lib = _load()
    A = _f64(A); B = _f64(B); gA = _f64(gA); gB = _f64(gB)
    gp = np.zeros(4); lam = np.zeros(2 * pr.n)
    if lib.oracle_adjoint(*pr._args(), _ptr(A), _ptr(B), _ptr(gA), _ptr(gB), _ptr(gp), _ptr(lam),
                          nthreads):
        raise ValueError("adjoint failed")
    return gp, lam


def condensate(pr: Problem, A, B) -> float:
    """Grid-truncated -<qbar q> = N_c/(4 pi^2) sum_j W_j B_j/(Q_j A_j^2 + B_j^2), N_c = 3."""
    lib = _load()
    A = _f64(A); B = _f64(B)
    return lib.oracle_condensate(pr.n, pr.s_min, pr.s_max, pr.grid_mode, _ptr(A), _ptr(B))


def max_threads() -> int:
    return _load().oracle_num_threads_available()
