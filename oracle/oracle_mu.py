"""FP64 CPU oracle of one sweep of the quark gap equation at finite chemical potential mu.

TEST INFRASTRUCTURE ONLY.  ``qdse_oracle_mu.cpp`` (plain C++ loops, explicit 4x4 complex Dirac
matrices) is the independent checker for a finite-mu solver; this module compiles it with the
host ``g++`` and wraps its C interface.  Only the test-suite may import it.  It imports nothing
from the GPU package.

The paper (arXiv:2012.03667) announces the finite-mu extension in Sec. V without giving its
equations; the readings M1-M5 taken for it are listed in the header of ``qdse_oracle_mu.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qdse_oracle_mu.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_mu.so")
_lib = None
_lock = threading.Lock()
_dp = ctypes.POINTER(ctypes.c_double)

BC, RL = 0, 1


def build(force: bool = False) -> str:
    """Compile into ``oracle/_build/liboracle_mu.so`` (host g++, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["g++", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", tmp, _SRC],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_mu_vertex.argtypes = ([_dp, ctypes.c_double, ctypes.c_double, _dp,
                                               ctypes.c_double, ctypes.c_double, _dp, _dp,
                                               ctypes.c_int, _dp, _dp, _dp])
            lib.oracle_mu_vertex.restype = None
            lib.oracle_mu_sweep.argtypes = ([ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp, _dp,
                                              ctypes.c_int, _dp, _dp] + [ctypes.c_double] * 5
                                             + [ctypes.c_int] + [_dp] * 9 + [ctypes.c_int])
            lib.oracle_mu_sweep.restype = ctypes.c_int
            _lib = lib
        return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _c(x):
    """Complex array -> interleaved float64."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).view(np.float64)


def _p(x):
    return x.ctypes.data_as(_dp)


def vertex(q, q4, p, p4, fq, fp, vertex=BC):
    """The vertex Gamma_nu(q~, p~) (reading M3; nu = 0..3) and S^-1(q~), S^-1(p~) as complex
    4x4 matrices.  q, p: spatial 3-vectors; q4, p4: complex fourth components (p_4 + i mu);
    fq, fp: (A, C, B) at q~ and p~."""
    lib = _load()
    gam = np.zeros(2 * 64); sq = np.zeros(32); sp = np.zeros(32)
    qa, pa = _f64(q), _f64(p)
    fqa, fpa = _c(fq), _c(fp)
    lib.oracle_mu_vertex(_p(qa), complex(q4).real, complex(q4).imag, _p(pa), complex(p4).real,
                         complex(p4).imag, _p(fqa), _p(fpa), vertex, _p(gam), _p(sq), _p(sp))
    return (gam.view(np.complex128).reshape(4, 4, 4), sq.view(np.complex128).reshape(4, 4),
            sp.view(np.complex128).reshape(4, 4))


def sweep(pv, p4, qv, q4, wq, z, wz, D, omega, m, mu, Ap, Cp, Bp, Aq, Cq, Bq, cf=4.0 / 3.0,
          vertex=BC, nthreads=0):
    """One finite-mu sweep (readings M1-M5): new (A, C, B) at the external points (|p_vec|, p_4)
    from the inputs there and at the internal points (|q_vec|, q_4) with weights wq (including
    |q|^2 d|q| dq_4) and cosine nodes z, wz."""
    lib = _load()
    pv, p4, qv, q4, wq, z, wz = map(_f64, (pv, p4, qv, q4, wq, z, wz))
    ins = [_c(x) for x in (Ap, Cp, Bp, Aq, Cq, Bq)]
    outs = [np.zeros(2 * len(pv)) for _ in range(3)]
    bad = lib.oracle_mu_sweep(len(pv), _p(pv), _p(p4), len(qv), _p(qv), _p(q4), _p(wq), len(z),
                              _p(z), _p(wz), D, omega, m, mu, cf, vertex, *[_p(x) for x in ins],
                              *[_p(x) for x in outs], nthreads)
    if bad:
        raise ValueError("singular propagator or k^2 = 0 at some (p, q) pair")
    return tuple(o.view(np.complex128) for o in outs)
