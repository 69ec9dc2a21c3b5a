"""Quadrature weights of the finite-mu grids: the caller's side of qdse_mu_grid_create.

The library takes the internal points' weights and the angular rule as inputs (include/qdse_mu.h).
This module forms them for grids whose |q| and |q_4| nodes are Gauss-Legendre nodes log-mapped onto
[lo, hi] and whose cosine nodes are Gauss-Legendre nodes on [-1, 1]:
  - int_lo^hi f(x) dx = int f(e^u) e^u du, so a node x_j carries (hi-lo in u)/2 v_j x_j;
  - the finite-mu measure d^4q/(2 pi)^4 = 2 pi/(2 pi)^4 dq_4 |q|^2 d|q| dz (the azimuth gives 2 pi;
    the constant is applied by the library) gives the internal point (|q|_r, q_4f) the weight
    w(|q|_r) |q|_r^2 w(|q_4f|), q_4 < 0 mirroring q_4 > 0.
At temperature T the fourth components are the fermion Matsubara frequencies q_4 = (2n + 1) pi T and
int dq_4/(2 pi) is T sum_n, so each frequency carries dq_4 = 2 pi T (matsubara_weights).
Host-side set-up of the grid (like the vacuum grid of csrc/grid.cpp); none of the sweep.
"""
from __future__ import annotations

import numpy as np


def log_gl_weights(x, lo: float, hi: float) -> np.ndarray:
    """dx weights of len(x) Gauss-Legendre nodes log-mapped onto [lo, hi]; x must be those nodes
    in ascending order."""
    x = np.asarray(x, dtype=np.float64)
    t, v = np.polynomial.legendre.leggauss(len(x))
    a, b = np.log(lo), np.log(hi)
    expect = np.exp(a + 0.5 * (t + 1.0) * (b - a))
    if not np.allclose(x, expect, rtol=1e-12, atol=0.0):
        raise ValueError("nodes are not Gauss-Legendre nodes log-mapped onto [lo, hi]")
    return 0.5 * (b - a) * v * x


def measure_weights(q_abs, q4, lo: float, hi: float) -> np.ndarray:
    """Weights w_q[r * len(q4) + f] = w(|q|_r) |q|_r^2 w(|q_4f|) of the internal product grid."""
    q_abs = np.asarray(q_abs, dtype=np.float64)
    q4 = np.asarray(q4, dtype=np.float64)
    pos = np.unique(np.abs(q4))
    w4 = log_gl_weights(pos, lo, hi)[np.searchsorted(pos, np.abs(q4))]
    return np.outer(log_gl_weights(q_abs, lo, hi) * q_abs ** 2, w4).ravel()


def angular_weights(z) -> np.ndarray:
    """Weights of int_{-1}^{1} dz on len(z) Gauss-Legendre nodes z (ascending)."""
    z = np.asarray(z, dtype=np.float64)
    t, v = np.polynomial.legendre.leggauss(len(z))
    if not np.allclose(z, t, rtol=0.0, atol=1e-14):
        raise ValueError("cosine nodes are not Gauss-Legendre nodes")
    return v


def matsubara_weights(q_abs, q4, T: float, lo: float, hi: float) -> np.ndarray:
    """Weights w_q[r * len(q4) + f] = w(|q|_r) |q|_r^2 2 pi T of the internal product grid at
    temperature T, whose q4 are fermion Matsubara frequencies (2n + 1) pi T of either sign."""
    q_abs = np.asarray(q_abs, dtype=np.float64)
    q4 = np.asarray(q4, dtype=np.float64)
    if not T > 0.0:
        raise ValueError("temperature must be positive")
    n = (np.abs(q4) / (np.pi * T) - 1.0) / 2.0
    if not np.allclose(n, np.round(n), rtol=0.0, atol=1e-9) or np.any(np.round(n) < 0):
        raise ValueError("q4 nodes are not fermion Matsubara frequencies of T")
    return np.outer(log_gl_weights(q_abs, lo, hi) * q_abs ** 2,
                    np.full(len(q4), 2.0 * np.pi * T)).ravel()
