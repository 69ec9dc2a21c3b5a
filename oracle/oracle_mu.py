"""FP64 CPU oracle of the quark gap equation at finite chemical potential mu: one sweep, the
interpolation onto the internal points, and the solve.

TEST INFRASTRUCTURE ONLY.  ``qdse_oracle_mu.cpp`` (plain C++ loops, explicit 4x4 complex Dirac
matrices) is the independent checker for a finite-mu solver; this module compiles it with the
host ``g++`` and wraps its C interface.  Only the test-suite may import it.  It imports nothing
from the GPU package.

The paper (arXiv:2012.03667) announces the finite-mu extension in Sec. V without giving its
equations.  Readings M1-M5 (the equation, vertex, projections and measure) are listed in the header
of ``qdse_oracle_mu.cpp``; M6 (interpolation onto the internal points), M7 (the iteration and its
convergence test) and M8 (the optional ray-blended difference quotient) are stated in
``interpolate``, ``solve`` and ``solve``'s ``ray_eta`` below.  The quadrature weights the oracle
sums with (reading M5's measure and the cosine rule) are formed here from the node arrays alone
(``measure``, ``angular_weights``: interpolatory rules from the moment equations), independently
of the weights the library is given.  Finite temperature (Sec. V names it as future work) is the
same sweep and solve on a grid whose fourth components are Matsubara frequencies, with the
Matsubara sum as the q_4 rule (readings T1, T2 in ``matsubara_measure``).
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
            lib.oracle_mu_sweep_dq.argtypes = ([ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp,
                                                 _dp, ctypes.c_int, _dp, _dp]
                                                + [ctypes.c_double] * 5 + [ctypes.c_int]
                                                + [_dp] * 10 + [ctypes.c_int])
            lib.oracle_mu_sweep_dq.restype = ctypes.c_int
            _lib = lib
        return _lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _c(x):
    """Complex array -> interleaved float64."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).view(np.float64)


def _p(x):
    return x.ctypes.data_as(_dp)


def interpolatory_weights(t):
    """Weights of the interpolatory rule on the nodes t (in (-1, 1), distinct): the w with
    sum_j w_j f(t_j) = int_{-1}^{1} f exactly for every polynomial of degree < len(t), from the
    moment equations sum_j w_j P_k(t_j) = int P_k = 2 [k = 0] in the Legendre basis (Bonnet's
    recurrence).  On Gauss-Legendre nodes these are the Gauss weights, exact to degree 2n - 1."""
    t = np.asarray(t, dtype=np.float64)
    n = len(t)
    V = np.empty((n, n))
    V[0] = 1.0
    if n > 1:
        V[1] = t
    for k in range(1, n - 1):
        V[k + 1] = ((2 * k + 1) * t * V[k] - k * V[k - 1]) / (k + 1)
    rhs = np.zeros(n)
    rhs[0] = 2.0
    return np.linalg.solve(V, rhs)


def log_rule(x, lo, hi):
    """Weights of int_lo^hi f(x) dx on nodes x that carry an interpolatory rule in u = ln x on
    [ln lo, ln hi] (dx = x du)."""
    x = np.asarray(x, dtype=np.float64)
    a, b = np.log(lo), np.log(hi)
    t = (2.0 * np.log(x) - (a + b)) / (b - a)
    return interpolatory_weights(t) * 0.5 * (b - a) * x


def measure(q_abs, q4, lo, hi):
    """Reading M5: the weights w_q of int |q|^2 d|q| dq_4 on the product grid q_abs x q4
    (row-major, point r * len(q4) + f), built here from the node arrays alone: |q| and |q_4| carry
    rules in ln x on [lo, hi] (log_rule); q_4 < 0 nodes mirror q_4 > 0 ones with their weights."""
    q_abs = np.asarray(q_abs, dtype=np.float64)
    q4 = np.asarray(q4, dtype=np.float64)
    pos = np.unique(np.abs(q4))
    w4p = log_rule(pos, lo, hi)
    w4 = w4p[np.searchsorted(pos, np.abs(q4))]
    wr = log_rule(q_abs, lo, hi) * q_abs ** 2
    return np.outer(wr, w4).ravel()


def angular_weights(z):
    """Weights of int_{-1}^{1} dz on the cosine nodes z (interpolatory rule)."""
    return interpolatory_weights(z)


def matsubara_measure(q_abs, q4, T, lo, hi):
    """Reading T1 (finite temperature, announced in Sec. V without equations): in the imaginary-time
    formalism the quark's fourth momentum takes the fermion Matsubara values q_4 = (2n + 1) pi T
    and int dq_4/(2 pi) becomes T sum_n, so reading M5's dq_4 becomes 2 pi T per frequency.  The
    weights w_q of int |q|^2 d|q| dq_4 on the product grid q_abs x q4 (row-major, point
    r * len(q4) + f) are then w(|q|_r) |q|_r^2 * 2 pi T, the radial rule in ln x on [lo, hi]
    (log_rule).  Every q4 must be an odd multiple of pi T (both signs); reading T2 truncates the
    sum to the frequencies given."""
    q_abs = np.asarray(q_abs, dtype=np.float64)
    q4 = np.asarray(q4, dtype=np.float64)
    if not T > 0.0:
        raise ValueError("temperature must be positive")
    k = q4 / (np.pi * T)
    odd = np.round((k - 1.0) / 2.0) * 2.0 + 1.0
    if not np.allclose(k, odd, rtol=0.0, atol=1e-9):
        raise ValueError("q4 nodes are not fermion Matsubara frequencies of T")
    wr = log_rule(q_abs, lo, hi) * q_abs ** 2
    return np.outer(wr, np.full(len(q4), 2.0 * np.pi * T)).ravel()


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
          vertex=BC, nthreads=0, Fd=None):
    """One finite-mu sweep (readings M1-M5): new (A, C, B) at the external points (|p_vec|, p_4)
    from the inputs there and at the internal points (|q_vec|, q_4) with weights wq (including
    |q|^2 d|q| dq_4) and cosine nodes z, wz.  Fd (reading M8): None, or complex [3, n_ext * n_int]
    -- per pair, the values subtracted in the vertex's difference numerators in place of the
    external point's own."""
    lib = _load()
    pv, p4, qv, q4, wq, z, wz = map(_f64, (pv, p4, qv, q4, wq, z, wz))
    ins = [_c(x) for x in (Ap, Cp, Bp, Aq, Cq, Bq)]
    outs = [np.zeros(2 * len(pv)) for _ in range(3)]
    if Fd is None:
        bad = lib.oracle_mu_sweep(len(pv), _p(pv), _p(p4), len(qv), _p(qv), _p(q4), _p(wq),
                                  len(z), _p(z), _p(wz), D, omega, m, mu, cf, vertex,
                                  *[_p(x) for x in ins], *[_p(x) for x in outs], nthreads)
    else:
        fd = _c(np.asarray(Fd).reshape(3, len(pv) * len(qv)))
        bad = lib.oracle_mu_sweep_dq(len(pv), _p(pv), _p(p4), len(qv), _p(qv), _p(q4), _p(wq),
                                     len(z), _p(z), _p(wz), D, omega, m, mu, cf, vertex,
                                     *[_p(x) for x in ins], _p(fd), *[_p(x) for x in outs],
                                     nthreads)
    if bad:
        raise ValueError("singular propagator or k^2 = 0 at some (p, q) pair")
    return tuple(o.view(np.complex128) for o in outs)


def interpolate(p_axis, p4_axis, F, q_abs, q4):
    """Values at the internal points of the product grid (q_abs x q4, row-major) from values F
    [3, n_pr * n_p4] on the external product grid (p_axis x p4_axis, row-major, both ascending,
    p4 > 0) -- reading M6: the staggered-grid rule of Sec. III applied along each axis in turn
    (linear in |p| and in p_4 between the bracketing nodes, held constant beyond the last node),
    and F(|q|, -q_4) = conj F(|q|, q_4) for q_4 < 0."""
    F = np.asarray(F, dtype=np.complex128).reshape(3, len(p_axis), len(p4_axis))

    def bracket(axis, x):
        # (lower index, weight of the upper node); x below the first node is held at it
        i = np.searchsorted(axis, x, side="right") - 1
        if i < 0:
            return 0, 0.0
        if i >= len(axis) - 1:
            return len(axis) - 1, 0.0
        return i, (x - axis[i]) / (axis[i + 1] - axis[i])

    out = np.empty((3, len(q_abs), len(q4)), dtype=np.complex128)
    for r, Q in enumerate(q_abs):
        i, a = bracket(p_axis, Q)
        i1 = min(i + 1, len(p_axis) - 1)
        for f, x4 in enumerate(q4):
            k, b = bracket(p4_axis, abs(x4))
            k1 = min(k + 1, len(p4_axis) - 1)
            v = ((1 - a) * (1 - b) * F[:, i, k] + a * (1 - b) * F[:, i1, k]
                 + (1 - a) * b * F[:, i, k1] + a * b * F[:, i1, k1])
            out[:, r, f] = np.conj(v) if x4 < 0 else v
    return out.reshape(3, -1)


def interpolate_points(p_axis, p4_axis, F, x, y):
    """Reading M6 at arbitrary points (|p| = x, p_4 = y; arrays of one shape), vectorised: the
    same bracketing, weights, holding and conjugation (y < 0) as interpolate().  Returns
    [3, *x.shape]."""
    F = np.asarray(F, dtype=np.complex128).reshape(3, len(p_axis), len(p4_axis))
    x = np.asarray(x, dtype=np.float64)
    ya = np.abs(np.asarray(y, dtype=np.float64))

    def bracket(axis, v):
        i = np.searchsorted(axis, v, side="right") - 1
        inside = (i >= 0) & (i < len(axis) - 1)
        ic = np.clip(i, 0, len(axis) - 1)
        i1 = np.minimum(ic + 1, len(axis) - 1)
        span = np.where(inside, axis[i1] - axis[ic], 1.0)
        w = np.where(inside, (v - axis[ic]) / span, 0.0)
        return ic, i1, w

    i, i1, a = bracket(np.asarray(p_axis), x)
    k, k1, b = bracket(np.asarray(p4_axis), ya)
    v = ((1 - a) * (1 - b) * F[:, i, k] + a * (1 - b) * F[:, i1, k]
         + (1 - a) * b * F[:, i, k1] + a * b * F[:, i1, k1])
    return np.where(np.asarray(y) < 0, np.conj(v), v)


def solve(p_axis, p4_axis, q_abs, q4, w_q, z, wz, D, omega, m, mu, F0, tol=1e-10, max_iter=500,
          cf=4.0 / 3.0, vertex=BC, alpha=1.0, nthreads=0, ray_eta=None):
    """Successive approximation (the paper's Eq. jifen14 scheme) of the finite-mu equation on the
    external product grid: G = sweep(F, interpolate(F)), F <- G (alpha = 1) or
    F <- (1 - alpha) F + alpha G, until the relative change of reading M7 (per function,
    max |F_new - F_old| over the grid divided by max |F_new|) is below tol; tol = 0 runs exactly
    max_iter steps.  (The change of a function that is identically zero is taken absolute.)

    ray_eta (reading M8, off when None): the difference numerators F_q - F_p of the vertex take,
    per pair, F_p + beta (F_ray - F_p) in place of F_p, where F_ray is F interpolated (M6) at the
    point of q's ray with p's 4-radius, (|q|, q_4) sqrt(P^2 + p_4^2)/sqrt(Q^2 + q_4^2), and
    beta = exp(-(2 mu |q_4 - p_4| / ray_eta)^2), ray_eta in GeV^2.  At mu = 0 the numerator then
    vanishes on the 4-sphere q^2 = p^2 for any grid function, so the discrete principal-value sum
    of 1/(q~^2 - p~^2) no longer couples F_p to itself; where 2 mu |q_4 - p_4| >> ray_eta it is
    the exact quotient of M3.
    Returns (F [3, n_ext], iterations, converged)."""
    PR, P4 = np.meshgrid(p_axis, p4_axis, indexing="ij")
    pv, p4 = PR.ravel(), P4.ravel()
    QR, Q4 = np.meshgrid(q_abs, q4, indexing="ij")
    qv, q4f = QR.ravel(), Q4.ravel()
    F = np.asarray(F0, dtype=np.complex128).reshape(3, -1).copy()
    if ray_eta is not None:
        lam = np.sqrt(pv ** 2 + p4 ** 2)[:, None] / np.sqrt(qv ** 2 + q4f ** 2)[None, :]
        rx, ry = qv[None, :] * lam, q4f[None, :] * lam
        beta = np.exp(-(2.0 * mu * np.abs(q4f[None, :] - p4[:, None]) / ray_eta) ** 2)
    for it in range(1, max_iter + 1):
        Fi = interpolate(p_axis, p4_axis, F, q_abs, q4)
        Fd = None
        if ray_eta is not None:
            Fr = interpolate_points(p_axis, p4_axis, F, rx, ry)
            Fp = F[:, :, None]
            Fd = (Fp + beta[None] * (Fr - Fp)).reshape(3, -1)
        G = np.array(sweep(pv, p4, qv, q4f, w_q, z, wz, D, omega, m, mu, *F, *Fi, cf=cf,
                           vertex=vertex, nthreads=nthreads, Fd=Fd))
        new = G if alpha == 1.0 else (1.0 - alpha) * F + alpha * G
        change = 0.0
        for c in range(3):
            d, mag = np.abs(new[c] - F[c]).max(), np.abs(new[c]).max()
            change = max(change, d / mag if mag > 0 else d)
        F = new
        if change < tol:
            return F, it, True
    return F, max_iter, False
