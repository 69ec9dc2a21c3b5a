"""Pins of the finite-temperature readings of the FP64 oracle (``oracle_mu.matsubara_measure`` with
the finite-mu sweep) against what the mathematics fixes (no GPU needed).

The paper names finite temperature as future work (Sec. V) and gives no equations.  Readings T1 and
T2 (``oracle_mu.matsubara_measure``): the fourth momentum runs over the fermion Matsubara
frequencies (2n + 1) pi T, int dq_4/(2 pi) -> T sum_n, the rest of the finite-mu equation
unchanged.  What pins them:
  * Poisson summation: for a Gaussian the frequency sum has a closed form whose alternating signs
    exist only for odd frequencies (even ones, or a missing 2 pi, fail by O(1));
  * the fermion sum of a free propagator, T sum_n 1/(w_n^2 + E^2) = tanh(E/2T)/(2E);
  * T -> 0: the whole Ball-Chiu sweep on Matsubara frequencies equals the sweep with the q_4
    integral done by a dense Gauss-Legendre rule, up to corrections exp(-d/T) set by the distance d
    of the integrand's nearest complex singularity in q_4.
"""
import numpy as np
import pytest

from oracle import oracle_mu as OM


def _odd(T, n):
    w = (2.0 * np.arange(n) + 1.0) * np.pi * T
    return np.concatenate([-w[::-1], w])


def _q4_weights(q4, T):
    """The q_4 factor of the oracle's product measure (one radial node, unit radial weight)."""
    q = np.array([1.0])
    wr = OM.log_rule(q, 0.5, 2.0) * q ** 2
    return OM.matsubara_measure(q, q4, T, 0.5, 2.0) / wr[0]


@pytest.mark.parametrize("T", [0.05, 0.15, 0.4])
def test_matsubara_measure_sums_a_gaussian_to_its_poisson_closed_form(T):
    """sum_f w_f exp(-q4_f^2/a) over the fermion frequencies = sqrt(pi a) sum_k (-1)^k
    exp(-a k^2/(4 T^2)) (Poisson summation of the half-shifted lattice).  With a = 4 T^2 the k = +-1
    terms carry 74% of the value, with the sign only odd frequencies give."""
    a = 4.0 * T * T
    q4 = _odd(T, 60)
    got = np.sum(_q4_weights(q4, T) * np.exp(-q4 ** 2 / a))
    k = np.arange(-30, 31)
    exact = np.sqrt(np.pi * a) * np.sum((-1.0) ** np.abs(k) * np.exp(-a * k ** 2 / (4 * T * T)))
    assert abs(got - exact) < 1e-13 * abs(exact)
    even = (2.0 * np.pi * T) * np.sum(np.exp(-((2.0 * np.arange(-60, 61)) * np.pi * T) ** 2 / a))
    assert abs(even - exact) > 0.5 * abs(exact)


def test_matsubara_measure_gives_the_fermion_sum_of_a_free_propagator():
    """T sum_n 1/(w_n^2 + E^2) = tanh(E/(2T))/(2E) (the weights carry dq_4 = 2 pi T, so the sum
    is the weighted sum over 2 pi); the truncated tail, 1/(pi^2 T) sum_{n >= N} (2/(2n+1)^2), is
    added back to third order.  E/T from 0.5 to 20."""
    T = 0.1
    N = 20000
    q4 = _odd(T, N)
    w = _q4_weights(q4, T)
    tail_n = 1.0 / (2.0 * (2 * N + 1)) + 1.0 / (2.0 * (2 * N + 1) ** 2)  # sum_{n>=N} 1/(2n+1)^2
    for E in (0.05, 0.3, 2.0):
        got = np.sum(w / (q4 ** 2 + E * E)) / (2.0 * np.pi) + 2.0 * tail_n / (np.pi ** 2 * T)
        exact = np.tanh(E / (2.0 * T)) / (2.0 * E)
        assert abs(got - exact) < 1e-10 * exact, (E, got, exact)


def test_matsubara_measure_refuses_frequencies_that_are_not_fermionic():
    with pytest.raises(ValueError):
        OM.matsubara_measure(np.array([1.0]), 2.0 * np.pi * 0.1 * np.arange(1, 4), 0.1, 0.5, 2.0)
    with pytest.raises(ValueError):
        OM.matsubara_measure(np.array([1.0]), _odd(0.1, 3), 0.0, 0.5, 2.0)


def _af(s):
    return 1 + 0.6 / (1 + s / 0.5)


def _bf(s, m):
    return 0.5 / (1 + s / 0.8) + m


def _fields(v, v4, m):
    s = v ** 2 + v4 ** 2
    return _af(s), 1.05 * _af(s), _bf(s, m)


def _composite_gl(edges, n):
    """Composite n-point Gauss-Legendre rule on consecutive panels [edges[k], edges[k+1]]."""
    t, v = np.polynomial.legendre.leggauss(n)
    x, w = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        x.append(0.5 * (b - a) * t + 0.5 * (a + b))
        w.append(0.5 * (b - a) * v)
    return np.concatenate(x), np.concatenate(w)


def test_low_temperature_bc_sweep_equals_the_continuum_q4_integral():
    """At low T the Ball-Chiu sweep with the Matsubara measure equals the same sweep with int dq_4
    done by a composite Gauss-Legendre rule, at the same external points (|p| between the internal
    |q| nodes, p_4 = the first three frequencies), with inputs analytic in q^2 (so the vertex's
    difference quotients stay finite).  As a function of q_4 the integrand is analytic except
    where the Landau projector's k^2 vanishes, q_4 = p_4 +- i |p_vec - q_vec| (|p_vec - q_vec| >=
    0.1375 GeV here), and at the propagator's zeros (about 0.3 GeV off the axis); so the Matsubara
    sum at T = 0.005 GeV (320 frequencies, up to 10 GeV) differs from the integral by about
    exp(-0.1375/T) ~ 1e-12 of the self-energy.  The continuum rule uses panels of 0.05 GeV near
    q_4 = 0 so that those singularities cost it nothing.  Required agreement: 1e-9.  A dropped
    2 pi in the measure fails by a factor 2 pi; T instead of 2 pi T likewise."""
    T, m = 0.005, 0.005
    lo, hi = 1e-2, 1e2
    t, _ = np.polynomial.legendre.leggauss(12)
    qr = np.exp(np.log(lo) + 0.5 * (t + 1) * (np.log(hi) - np.log(lo)))
    mid = np.sqrt(qr[:-1] * qr[1:])
    pa = mid[(mid > 0.2) & (mid < 4.0)]
    assert min(np.abs(p - qr).min() for p in pa) > 0.137
    wn = (2.0 * np.arange(320) + 1.0) * np.pi * T
    q4m = np.concatenate([-wn[::-1], wn])
    wr = OM.log_rule(qr, lo, hi) * qr ** 2
    wqm = OM.matsubara_measure(qr, q4m, T, lo, hi)
    half = np.concatenate([np.linspace(0.0, 1.0, 21), np.linspace(1.25, 3.0, 8),
                           np.arange(4.0, 13.0, 1.0)])
    q4c, w4c = _composite_gl(np.concatenate([-half[::-1], half[1:]]), 12)
    wqc = np.outer(wr, w4c).ravel()
    z, wz = np.polynomial.legendre.leggauss(16)
    PR, P4 = np.meshgrid(pa, wn[:3], indexing="ij")
    pv, p4 = PR.ravel(), P4.ravel()
    Fe = _fields(pv, p4, m)
    out = []
    for q4, wq in ((q4m, wqm), (q4c, wqc)):
        QR, Q4 = np.meshgrid(qr, q4, indexing="ij")
        Fi = _fields(QR.ravel(), Q4.ravel(), m)
        out.append(np.array(OM.sweep(pv, p4, QR.ravel(), Q4.ravel(), wq, z, wz, 0.55, 0.678, m,
                                     0.0, *Fe, *Fi, vertex=OM.BC, nthreads=0)))
    x0 = np.array([1.0, 1.0, m])[:, None]
    scale = np.abs(out[1] - x0).max(axis=1)
    err = (np.abs(out[0] - out[1]).max(axis=1) / scale).max()
    assert err < 1e-9, err
    assert np.abs(out[0].imag).max() < 1e-13  # mu = 0: the +-w_n pairs cancel the imaginary parts
