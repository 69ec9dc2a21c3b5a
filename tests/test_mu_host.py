"""The finite-mu pair arithmetic of the CUDA path (csrc/mu_pair.cuh: moments, stored planes,
propagator parts, per-pair closed-form traces) against the FP64 oracle, on the CPU.

``tests/mu/host_mu_sweep.cpp`` compiles that header with the host g++ and sums every pair in plain
loops (no windows, no GPU), in FP64 and in FP32.  The oracle computes the same sweep with explicit
4x4 complex Dirac matrices, so agreement pins the closed-form traces the kernels use.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle_mu as OM
from paper_2012_03667_gb300 import inputs as I
from paper_2012_03667_gb300 import mu_rule as MR

def gpu_rule(w):
    """The library's quadrature inputs for workload w: internal weights, cosine nodes and weights
    (formed on the package side, paper_2012_03667_gb300/mu_rule.py)."""
    return MR.measure_weights(w.q_abs, w.q4, w.lo, w.hi), w.z, MR.angular_weights(w.z)


def oracle_rule(w):
    """The oracle's own weights for the same nodes (reading M5, interpolatory rules)."""
    return OM.measure(w.q_abs, w.q4, w.lo, w.hi), w.z, OM.angular_weights(w.z)


HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mu", "host_mu_sweep.cpp")
HDR = os.path.join(HERE, "..", "paper_2012_03667_gb300", "csrc", "mu_pair.cuh")
LIB = os.path.join(HERE, "mu", "_build", "libhostmu.so")
_dp = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def host():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                               os.path.getmtime(HDR))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, SRC], check=True)
        os.replace(tmp, LIB)
    lib = ctypes.CDLL(LIB)
    lib.host_mu_sweep.restype = None
    lib.host_mu_sweep.argtypes = ([ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp, _dp,
                                   ctypes.c_int, _dp, _dp] + [ctypes.c_double] * 5
                                  + [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp])

    def run(pv, p4, qv, q4, wq, z, wz, D, om, m, mu, Fp, Fq, rainbow, fp32):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (pv, p4, qv, q4, wq, z, wz)]
        Fp = np.ascontiguousarray(np.asarray(Fp, dtype=np.complex128)).view(np.float64)
        Fq = np.ascontiguousarray(np.asarray(Fq, dtype=np.complex128)).view(np.float64)
        Fo = np.zeros(6 * len(pv))
        p = lambda a: a.ctypes.data_as(_dp)
        lib.host_mu_sweep(len(pv), p(arrs[0]), p(arrs[1]), len(qv), p(arrs[2]), p(arrs[3]),
                          p(arrs[4]), len(z), p(arrs[5]), p(arrs[6]), D, om, m, mu, 4.0 / 3.0,
                          rainbow, fp32, p(Fp), p(Fq), p(Fo))
        return Fo.view(np.complex128).reshape(3, len(pv))
    return run


def _workload():
    w = I.mu_workload(n_r=12, n_4=8, n_z=24, n_mu=3, mu_range=(0.0, 0.4))
    QR, Q4 = np.meshgrid(w.q_abs, w.q4, indexing="ij")
    return w, QR.ravel(), Q4.ravel()


@pytest.mark.parametrize("vertex", [OM.BC, OM.RL])
def test_pair_arithmetic_matches_the_oracle(host, vertex):
    """FP64 to 1e-12 and FP32 to 1e-4 of max |F - x0| (the self-energy part).  The FP32 bound is
    set by the BC difference quotients (F_q - F_p)/(q~^2 - p~^2) of rounded inputs near equal
    4-radii at small mu; observed 2e-5 on larger grids, 1e-6 elsewhere."""
    w, qv, q4 = _workload()
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for mu in list(w.mu) + [0.0]:
        Fp = I.mu_iterate(w.p_abs, w.p4, mu, w.m)
        Fq = I.mu_iterate(qv, q4, mu, w.m)
        ref = np.array(OM.sweep(w.p_abs, w.p4, qv, q4, *oracle_rule(w), w.D, w.omega, w.m, mu,
                                *Fp, *Fq, vertex=vertex))
        scale = np.abs(ref - x0).max(axis=1)
        assert np.all(scale > 1e-3)
        for fp32, tol in ((0, 1e-12), (1, 1e-4)):
            got = host(w.p_abs, w.p4, qv, q4, *gpu_rule(w), w.D, w.omega, w.m, mu, Fp, Fq,
                       vertex, fp32)
            err = (np.abs(got - ref).max(axis=1) / scale).max()
            assert err < tol, (mu, fp32, err)


def test_matsubara_workload_and_weights_on_the_package_side():
    """The finite-temperature workload's nodes are the fermion Matsubara frequencies (external p_4
    the positive ones, internal q_4 both signs), its external |p| never equal an internal |q|, and
    the package-side weights carry 2 pi T per frequency; frequencies of another T are refused."""
    T = 0.1
    w = I.matsubara_workload(T, n_r=8, n_4=4, n_z=8, n_mu=3)
    assert np.allclose(np.unique(w.p4), (2 * np.arange(4) + 1) * np.pi * T, rtol=1e-15)
    assert np.allclose(w.q4, np.concatenate([-np.unique(w.p4)[::-1], np.unique(w.p4)]))
    assert np.abs(np.unique(w.p_abs)[:, None] - w.q_abs[None, :]).min() > 0
    wq = MR.matsubara_weights(w.q_abs, w.q4, T, w.lo, w.hi).reshape(8, 8)
    wr = MR.log_gl_weights(w.q_abs, w.lo, w.hi) * w.q_abs ** 2
    assert np.allclose(wq, np.outer(wr, np.full(8, 2 * np.pi * T)), rtol=1e-15, atol=0)
    with pytest.raises(ValueError):
        MR.matsubara_weights(w.q_abs, w.q4 * 1.01, T, w.lo, w.hi)
    with pytest.raises(ValueError):
        MR.matsubara_weights(w.q_abs, w.q4, 0.0, w.lo, w.hi)
