"""The kernel precompute's double-float arithmetic (csrc/f2.cuh), compiled for the host, against
extended-precision evaluations of what it computes.

``tests/f2/host_f2.cpp`` compiles the header with the host g++.  The references are written here
from the definitions (numpy long double sums of the angular kernels with the g_3 numerator as
printed in Sec. II after the traces, exp of the long double argument), so they share nothing with
the header.  Tolerances: exp to 2e-14 relative; the entries K_0, K_T to 5e-14 relative and K_3 to
5e-14 of |K_T| + 3 sqrt(PQ) sum |w e z| (the magnitudes of the two sums it is the difference of).
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "f2", "host_f2.cpp")
HDR = os.path.join(HERE, "..", "paper_2012_03667_gb300", "csrc", "f2.cuh")
LIB = os.path.join(HERE, "f2", "_build", "libhostf2.so")
_dp = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                               os.path.getmtime(HDR))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                        tmp, SRC], check=True)
        os.replace(tmp, LIB)
    L = ctypes.CDLL(LIB)
    L.host_exp_neg.restype = ctypes.c_double
    L.host_exp_neg.argtypes = [ctypes.c_float, ctypes.c_float]
    L.host_pair_entries.restype = ctypes.c_int
    L.host_pair_entries.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_double, _dp]
    return L


def _f2(x):
    h = np.float32(x)
    return h, np.float32(np.float64(x) - np.float64(h))


def test_exp_of_a_pair_matches_long_double_exp(lib):
    rng = np.random.default_rng(11)
    d = np.concatenate([rng.uniform(0, 87.4, 4000), rng.uniform(0, 1e-3, 200), [0.0, 0.125,
                        0.25, 60.0, 87.4]])
    worst = 0.0
    for x in d:
        h, l = _f2(x)
        ref = np.exp(-(np.longdouble(h) + np.longdouble(l)))
        got = lib.host_exp_neg(h, l)
        # below exp(-75) the low float of the pair is subnormal: an absolute floor at the
        # subnormal spacing (the stored kernel pool has the same limit)
        worst = max(worst, float(abs(np.longdouble(got) - ref) / (ref + np.longdouble(1e-30))))
    assert worst < 2e-14, worst


PI_L = np.longdouble("3.14159265358979323846264338327950288")


def _chebyshev(nt):
    """Gauss-Chebyshev (2nd kind) nodes in long double: y = 1 - z = 2 sin^2(theta/2), z, 1 - z^2,
    weights; the harness gets their FP64 roundings."""
    th = np.arange(1, nt + 1, dtype=np.longdouble) * PI_L / (nt + 1)
    sn = np.sin(th)
    return 2 * np.sin(th / 2) ** 2, np.cos(th), sn ** 2, PI_L / (nt + 1) * sn ** 2


def _reference(P, Q, omega, nt):
    """Long double sums of the kernels' definition: K_n = 8 pi^2/w^4 sum_k w_k e^{-k^2/w^2} g_n,
    g_0 = 1, g_T = 2PQ(1 - z^2)/k^2, g_3 = [3x(P + Q) - 4x^2 - 2PQ]/k^2, x = sqrt(PQ) z."""
    L = np.longdouble
    y, z, s2, w = _chebyshev(nt)
    # sqrt P and sqrt Q as the FP64 grid holds them, and P, Q as their squares: the kernels are
    # functions of these rounded nodes, and the g_3 numerator, which cancels near the diagonal by
    # a factor up to 1e4, needs P and sqrt P consistent beyond FP64 rounding
    rP, rQ = L(np.sqrt(P)), L(np.sqrt(Q))
    P, Q, om = rP * rP, rQ * rQ, L(omega)
    k2 = (rP - rQ) ** 2 + 2 * rP * rQ * y
    e = w * np.exp(-k2 / om ** 2)
    x = rP * rQ * z
    pref = 8 * PI_L ** 2 / om ** 4
    K0 = pref * e.sum()
    KT = pref * (e * 2 * P * Q * s2 / k2).sum()
    g3n = 3 * x * (P + Q) - 4 * x * x - 2 * P * Q
    K3 = pref * (e * g3n / k2).sum()
    # K_3 = 3 sqrt(PQ) sum(w e z) - K_T: its condition is set by sum |w e z|
    scale3 = abs(KT) + abs(pref * 3 * rP * rQ * np.abs(e * z).sum())
    return K0, KT, K3, scale3


@pytest.mark.parametrize("nt", [32, 64, 128])
def test_pair_entries_match_long_double_sums(lib, nt):
    """Random pairs of the scan's grids (log-mapped nodes on [1e-4, 1e4], w in [0.4, 0.6]) inside
    the bands, including diagonal and neighbouring pairs where the g_3 numerator cancels."""
    rng = np.random.default_rng(nt)
    out = np.zeros(3)
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in _chebyshev(nt)]
    ptrs = [a.ctypes.data_as(_dp) for a in args]
    worst = [0.0, 0.0, 0.0]
    checked = 0
    for trial in range(300):
        om = rng.uniform(0.4, 0.6)
        P = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e4))))
        kind = trial % 3
        if kind == 0:
            Q = P
        elif kind == 1:
            Q = P * float(np.exp(rng.uniform(-0.1, 0.1)))
        else:
            Q = float((np.sqrt(P) + rng.uniform(-1, 1) * np.sqrt(70.0) * om) ** 2)
        if Q <= 0:
            continue
        kept = lib.host_pair_entries(P, Q, om, nt, *ptrs, 60.0, out.ctypes.data_as(_dp))
        K0, KT, K3, sc3 = _reference(P, Q, om, nt)
        if not kept:
            # stored as zeros: the first term is below the FP32 range
            assert float(K0) < 1e-30 * 8 * np.pi ** 2 / om ** 4 * 100
            continue
        checked += 1
        # floor: the FP32 range of the pair's low float times the kernels' scale 8 pi^2/w^4
        fl = 1e-30 * 8 * np.pi ** 2 / om ** 4
        worst[0] = max(worst[0], float(abs(out[0] - K0) / (K0 + fl)))
        worst[1] = max(worst[1], float(abs(out[1] - KT) / (KT + fl)))
        worst[2] = max(worst[2], float(abs(out[2] - K3) / (sc3 + fl)))
    assert checked > 100
    assert worst[0] < 5e-14 and worst[1] < 5e-14 and worst[2] < 5e-14, worst
