"""Pins of the finite-mu FP64 oracle (``oracle/qdse_oracle_mu.cpp``) against what the mathematics
fixes (no GPU needed).

The paper announces the finite chemical potential extension (Sec. V) without its equations; the
oracle takes readings M1-M5 (its header).  These tests pin it to things other than itself:
  * the Dirac algebra of its gamma matrices;
  * the Ward-Takahashi identity that defines the Ball-Chiu construction (M3), at complex momenta;
  * the chiral limit (B stays exactly zero) and the p_4 -> -p_4 conjugation symmetry;
  * the mu = 0 limit against the vacuum oracle, which is pinned on its own;
  * the contour-shift invariance at mu > 0: with inputs analytic in q~^2 and no propagator pole
    between Im q_4 = 0 and mu, the q_4 integral can be moved back to the real axis, so A, C, B
    depend on (|p_vec|, p_4, mu) only through p~^2 = p_vec^2 + (p_4 + i mu)^2, and C = A.
A slip in the mu terms (projecting C on p_4 instead of p~_4, dropping i mu from the vertex, the
wrong sign of mu) breaks the last one by at least 0.2, against a quadrature spread of 4e-4.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle import oracle_mu as OM

def oracle_rule(w):
    """The oracle's own weights for the same nodes (reading M5, interpolatory rules)."""
    return OM.measure(w.q_abs, w.q4, w.lo, w.hi), w.z, OM.angular_weights(w.z)


D, OMEGA, M = 0.93, 0.5, 0.005


def _gl(n):
    return np.polynomial.legendre.leggauss(n)


def _grid(nr, n4, a=0.5, R=60.0):
    """Internal points (|q_vec|, q_4) on a sinh-mapped Gauss-Legendre product rule covering
    |q_vec| in [0, R] and q_4 in [-R, R]; weights include |q_vec|^2 d|q_vec| dq_4.  The q_4 nodes
    are symmetric about 0."""
    U = np.arcsinh(R / a)
    t, w = _gl(nr)
    ur, wr = 0.5 * U * (t + 1), 0.5 * U * w
    qr = a * np.sinh(ur)
    jr = a * np.cosh(ur) * wr * qr ** 2
    t, w = _gl(n4)
    q4 = a * np.sinh(U * t)
    j4 = a * np.cosh(U * t) * U * w
    QR, Q4 = np.meshgrid(qr, q4, indexing="ij")
    WR, W4 = np.meshgrid(jr, j4, indexing="ij")
    return QR.ravel(), Q4.ravel(), (WR * W4).ravel()


def _af(s):
    return 1 + 0.6 / (1 + s / 0.5)


def _bf(s):
    return 0.5 / (1 + s / 0.8) + M


def _inputs(qv, q4, mu):
    s = qv ** 2 + (q4 + 1j * mu) ** 2
    return _af(s), _af(s), _bf(s)


def _rand_momenta(rng, mu):
    q, p = rng.normal(size=3), rng.normal(size=3)
    return q, complex(rng.normal(), mu), p, complex(rng.normal(), mu)


# --------------------------------------------------------------------------------------------
def test_gamma_matrices_are_hermitian_and_satisfy_the_clifford_algebra():
    rng = np.random.default_rng(1)
    q, q4, p, p4 = _rand_momenta(rng, 0.3)
    g, _, _ = OM.vertex(q, q4, p, p4, (1, 1, 0.3), (1, 1, 0.3), vertex=OM.RL)
    for a in range(4):
        np.testing.assert_allclose(g[a], g[a].conj().T, atol=0)
        for b in range(4):
            np.testing.assert_allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * (a == b) * np.eye(4),
                                       atol=1e-15)


@pytest.mark.parametrize("mu", [0.0, 0.25, 0.6])
def test_bc_vertex_satisfies_the_ward_takahashi_identity_at_complex_momenta(mu):
    """M3: i (q~ - p~)_nu Gamma_nu = S^-1(q~) - S^-1(p~), with complex A, C, B, C != A."""
    rng = np.random.default_rng(int(10 * mu) + 2)
    for _ in range(5):
        q, q4, p, p4 = _rand_momenta(rng, mu)
        fq = rng.normal(size=3) + 1j * rng.normal(size=3)
        fp = rng.normal(size=3) + 1j * rng.normal(size=3)
        g, sq, sp = OM.vertex(q, q4, p, p4, fq, fp)
        d = np.array([q[0] - p[0], q[1] - p[1], q[2] - p[2], q4 - p4])
        lhs = 1j * np.einsum("n,nab->ab", d, g)
        np.testing.assert_allclose(lhs, sq - sp, rtol=0, atol=1e-12 * np.abs(sq - sp).max())
        # the projections of M4 give back A, C, B from S^-1 of M1
        G = OM.vertex(q, q4, p, p4, fq, fp, vertex=OM.RL)[0]
        gq = np.einsum("k,kab->ab", q, G[:3])
        assert abs(np.trace(gq @ sq) / (4j * (q @ q)) - fq[0]) < 1e-13
        assert abs(np.trace(G[3] @ sq) / (4j * q4) - fq[1]) < 1e-13
        assert abs(np.trace(sq) / 4 - fq[2]) < 1e-13


def test_chiral_limit_keeps_B_exactly_zero():
    """m = 0 and B = 0 at every point: tr of an odd number of gamma matrices vanishes, so B stays 0
    (chiral symmetry) while A and C do not."""
    qv, q4, wq = _grid(16, 32)
    z, wz = _gl(12)
    mu = 0.2
    pv, p4 = np.array([0.3, 1.1]), np.array([0.2, -0.7])
    Aq, Cq, _ = _inputs(qv, q4, mu)
    Ap, Cp, _ = _inputs(pv, p4, mu)
    A, C, B = OM.sweep(pv, p4, qv, q4, wq, z, wz, D, OMEGA, 0.0, mu, Ap, Cp, 0 * Ap, Aq, Cq, 0 * Aq)
    assert np.all(np.abs(B) < 1e-15)
    assert np.all(np.abs(A - 1) > 1e-2) and np.all(np.abs(C - 1) > 1e-2)


@pytest.mark.parametrize("vertex", [OM.BC, OM.RL])
def test_reflecting_p4_conjugates_the_result(vertex):
    """With inputs F(q~^2) real-analytic and a q_4 rule symmetric about 0, p_4 -> -p_4 maps p~^2
    to its conjugate and the sweep output to its conjugate (to rounding)."""
    qv, q4, wq = _grid(16, 32)
    z, wz = _gl(12)
    mu = 0.3
    pv = np.array([0.4, 0.4, 1.3, 1.3])
    p4 = np.array([0.5, -0.5, 0.9, -0.9])
    Aq, Cq, Bq = _inputs(qv, q4, mu)
    Ap, Cp, Bp = _inputs(pv, p4, mu)
    out = OM.sweep(pv, p4, qv, q4, wq, z, wz, D, OMEGA, M, mu, Ap, Cp, Bp, Aq, Cq, Bq,
                   vertex=vertex)
    for F in out:
        assert np.abs(F.imag[0::2]).min() > 1e-4  # mu > 0 really makes the result complex
        np.testing.assert_allclose(F[1::2], F[0::2].conj(), rtol=1e-12, atol=0)


def test_mu_zero_reduces_to_the_vacuum_oracle():
    """At mu = 0 with C = A, real inputs: A = C and B agree with the vacuum sweep of the pinned
    vacuum oracle at its collocation nodes p^2 ~ 0.1 and 1 (point put off the 4-axis at angle 0.3),
    to the two quadratures' difference (below 2e-4 relative to A - 1 and B - m here)."""
    pr = O.Problem(n=128, n_theta=64, D=D, omega=OMEGA, m=M)
    sp, sq, _, _ = O.radial_grid(128)
    FA, FB = O.sweep(pr, _af(sq), _bf(sq), nthreads=O.max_threads())
    idx = [int(np.argmin(abs(sp - P))) for P in (0.1, 1.0)]
    P = sp[idx]
    pv, p4 = np.sqrt(P) * np.cos(0.3), np.sqrt(P) * np.sin(0.3)
    qv, q4, wq = _grid(48, 96)
    z, wz = _gl(24)
    Aq, Cq, Bq = _inputs(qv, q4, 0.0)
    A, C, B = OM.sweep(pv, p4, qv, q4, wq, z, wz, D, OMEGA, M, 0.0, _af(P), _af(P), _bf(P),
                       Aq, Cq, Bq, nthreads=O.max_threads())
    for F in (A, C, B):
        assert np.abs(F.imag).max() < 1e-14
    tol = 2e-3
    assert np.all(np.abs(A.real - FA[idx]) < tol * np.abs(FA[idx] - 1))
    assert np.all(np.abs(C.real - FA[idx]) < tol * np.abs(FA[idx] - 1))
    assert np.all(np.abs(B.real - FB[idx]) < tol * np.abs(FB[idx] - M))


@pytest.mark.parametrize("vertex", [OM.BC, OM.RL])
def test_result_depends_on_mu_only_through_p_tilde_squared(vertex):
    """Contour shift: three points (|p_vec|, p_4, mu) with mu = 0.05, 0.1, 0.2 and the same
    p~^2 = 0.73 + 0.04 i give the same A, C, B, and C = A.  The inputs' propagator pole sits at
    q~^2 = -0.109 (mass 0.33 > mu) and their own poles at q~^2 = -0.5 and -0.8, so the shift crosses
    none.  The spread is quadrature error: 2.3e-3, 3.4e-4, 1.1e-4 at 16, 24, 32 cosine nodes."""
    s = np.linspace(-0.49, -1e-6, 4000)
    disc = s * _af(s) ** 2 + _bf(s) ** 2
    s_pole = s[np.argmin(np.abs(disc))]
    assert -0.12 < s_pole < -0.10
    qv, q4, wq = _grid(48, 96)
    z, wz = _gl(24)
    c, d = 0.04, 0.73  # 2 p_4 mu = c, |p_vec|^2 + p_4^2 - mu^2 = d
    res = []
    for mu in (0.05, 0.1, 0.2):
        assert mu ** 2 < -s_pole
        p4 = c / (2 * mu)
        pv = np.sqrt(d - p4 ** 2 + mu ** 2)
        Ap, Cp, Bp = _inputs(np.array([pv]), np.array([p4]), mu)
        Aq, Cq, Bq = _inputs(qv, q4, mu)
        A, C, B = OM.sweep([pv], [p4], qv, q4, wq, z, wz, D, OMEGA, M, mu, Ap, Cp, Bp, Aq, Cq, Bq,
                           vertex=vertex, nthreads=O.max_threads())
        res.append((A[0], C[0], B[0]))
    res = np.array(res)
    assert abs(res[0, 0].imag) > 5e-3  # genuinely complex
    tol = 1e-3
    assert np.abs(res[:, 0] - res[0, 0]).max() < tol
    assert np.abs(res[:, 1] - res[:, 0]).max() < tol
    assert np.abs(res[:, 2] - res[0, 2]).max() < tol


def test_interpolation_is_exact_for_bilinear_functions_held_outside_and_mirrored():
    """Reading M6: linear in |p| and in p_4 between bracketing external nodes (so any function
    a + b|p| + c p_4 + d |p| p_4 is reproduced exactly inside the grid), held at the last node
    beyond it, and conjugated for q_4 < 0."""
    pa = np.array([0.1, 0.5, 1.0, 2.0])
    p4a = np.array([0.05, 0.4, 1.5])
    PR, P4 = np.meshgrid(pa, p4a, indexing="ij")

    def f(x, y):
        return (1 + 2j) + (0.3 - 0.1j) * x + (0.2 + 0.5j) * y + 0.7j * x * y

    F = np.array([f(PR, P4).ravel(), 2 * f(PR, P4).ravel(), -f(PR, P4).ravel()])
    qa = np.array([0.1, 0.2, 0.7, 1.9, 3.0])
    q4 = np.array([-1.0, -0.1, 0.05, 0.2, 1.2, 2.0])
    out = OM.interpolate(pa, p4a, F, qa, q4).reshape(3, len(qa), len(q4))
    for r, Q in enumerate(qa):
        for k, x4 in enumerate(q4):
            want = f(min(Q, 2.0), min(abs(x4), 1.5))
            want = np.conj(want) if x4 < 0 else want
            np.testing.assert_allclose(out[:, r, k], [want, 2 * want, -want], rtol=0, atol=1e-14)


def test_solve_reaches_a_fixed_point_of_the_sweep():
    """The solve (rainbow vertex, mu = 0.1, a coarse staggered grid) stops at a point where one
    more sweep moves every function by less than its tolerance, in the same number of steps from
    a damped iteration's limit; tol = 0 runs exactly max_iter steps."""
    from paper_2012_03667_gb300 import inputs as I
    w = I.mu_workload(n_r=12, n_4=8, n_z=24, n_mu=1)
    pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
    F0 = np.array([np.ones(len(w.p_abs)), np.ones(len(w.p_abs)), 0.3 * np.ones(len(w.p_abs))])
    args = (pa, p4a, w.q_abs, w.q4, *oracle_rule(w), w.D, w.omega, w.m, 0.1)
    F, it, ok = OM.solve(*args, F0, tol=1e-11, max_iter=200, vertex=OM.RL)
    assert ok and 10 < it < 100
    G, _, _ = OM.solve(*args, F, tol=0.0, max_iter=1, vertex=OM.RL)
    for c in range(3):
        assert np.abs(G[c] - F[c]).max() < 1e-10 * np.abs(F[c]).max()
    Fd, itd, okd = OM.solve(*args, F0, tol=1e-11, max_iter=400, vertex=OM.RL, alpha=0.7)
    assert okd and np.abs(Fd - F).max() < 1e-9 * np.abs(F).max()
    assert abs(F[0][0].imag) > 1e-4  # mu > 0: genuinely complex


def test_mu_zero_solve_approaches_the_vacuum_solution_as_the_grid_is_refined():
    """The whole finite-mu solve (sweep, interpolation M6, iteration M7) at mu = 0, rainbow
    vertex, against the pinned vacuum oracle's solve on its own 1-D grid: the 2-D solution is
    real, and its distance to the vacuum B(p^2) and the O(4) breaking |C - A| both shrink as the
    (|p|, p_4) grid is refined (observed: B 0.79 -> 0.19 of max|B|, |C - A| 1.05 -> 0.53, and
    0.055, 0.17 on a 24 x 16 grid).  It checks the pieces together, not each formula: a swap of
    the two interpolation weights still passes here and is caught by the exactness pin above."""
    from paper_2012_03667_gb300 import inputs as I
    pr = O.Problem(n=128, n_theta=64, D=D, omega=OMEGA, m=M, vertex=O.RL)
    A, B, it, ch, st = O.solve(pr, tol=1e-12, nthreads=O.max_threads())
    assert st == 0
    sp, _, _, _ = O.radial_grid(128)
    errs = []
    for nr, n4 in ((12, 8), (16, 12)):
        w = I.mu_workload(n_r=nr, n_4=n4, n_z=16, n_mu=1, D=D, omega=OMEGA, m=M)
        pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
        ones = np.ones(len(w.p_abs))
        F, it, ok = OM.solve(pa, p4a, w.q_abs, w.q4, *oracle_rule(w), D, OMEGA, M, 0.0,
                             np.array([ones, ones, 0.3 * ones]), tol=1e-10, max_iter=200,
                             vertex=OM.RL)
        assert ok and np.abs(F.imag).max() < 1e-13
        s = w.p_abs ** 2 + w.p4 ** 2
        sel = (s > 1e-3) & (s < 10)
        Bv = np.interp(np.log(s[sel]), np.log(sp), B)
        errs.append((np.abs(F[2].real[sel] - Bv).max() / np.abs(Bv).max(),
                     np.abs(F[1] - F[0]).max()))
    assert errs[1][0] < 0.5 * errs[0][0] and errs[1][0] < 0.3
    assert errs[1][1] < 0.7 * errs[0][1]


def test_vectorised_interpolation_and_the_m8_hook_reduce_to_the_plain_forms():
    """interpolate_points equals interpolate at the internal points (exactly); and a sweep whose
    difference numerators are handed the external point's own values (M8 with beta = 0) is
    bitwise the plain sweep."""
    from paper_2012_03667_gb300 import inputs as I
    w = I.mu_workload(n_r=8, n_4=6, n_z=12, n_mu=1)
    pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
    rng = np.random.default_rng(3)
    F = rng.normal(size=(3, len(w.p_abs))) + 1j * rng.normal(size=(3, len(w.p_abs)))
    QR, Q4 = np.meshgrid(w.q_abs, w.q4, indexing="ij")
    qv, q4 = QR.ravel(), Q4.ravel()
    Fi = OM.interpolate(pa, p4a, F, w.q_abs, w.q4)
    assert np.array_equal(OM.interpolate_points(pa, p4a, F, qv, q4), Fi)
    F = np.abs(F) + 0.5  # keep the propagator regular
    Fi = OM.interpolate(pa, p4a, F, w.q_abs, w.q4)
    args = (w.p_abs, w.p4, qv, q4, *oracle_rule(w), 0.55, 0.678, w.m, 0.13, *F, *Fi)
    plain = np.array(OM.sweep(*args))
    hooked = np.array(OM.sweep(*args, Fd=np.repeat(F, len(qv), axis=1)))
    assert np.array_equal(plain, hooked)


def test_ray_blended_quotient_converges_at_mu_zero_and_matches_the_exact_one_elsewhere():
    """Reading M8 (paper's interaction D = 0.55, omega = 0.678, BC vertex, 12 x 8 grid, start
    A = C = B = 1).  With the exact quotient of M3 one external point runs away at mu = 0 (its
    self-coupling through the discrete principal-value sum exceeds 1; A grows by 11% per sweep)
    and mu = 0.01 contracts by only 0.985 per sweep.  With the ray-blended quotient,
    ray_eta = 0.002, mu = 0 converges in about 40 sweeps; at mu = 0.2, where both converge, the
    solutions agree to 1e-4 (observed 2.1e-5; 8.9e-5 at mu = 0.1, 2.4e-4 at 0.05)."""
    from paper_2012_03667_gb300 import inputs as I
    w = I.mu_workload(n_r=12, n_4=8, n_z=16, n_mu=1, D=0.55, omega=0.678)
    pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
    start = np.array([np.ones(len(w.p_abs))] * 3, dtype=np.complex128)
    args = (pa, p4a, w.q_abs, w.q4, *oracle_rule(w), 0.55, 0.678, w.m)
    F0, it0, ok0 = OM.solve(*args, 0.0, start, tol=1e-10, max_iter=80, ray_eta=0.002,
                            nthreads=O.max_threads())
    assert ok0 and it0 <= 60
    assert np.abs(F0.imag).max() < 1e-13 and 0.4 < (F0[2][0] / F0[0][0]).real < 0.7
    Fr, itr, okr = OM.solve(*args, 0.2, start, tol=1e-10, max_iter=150, ray_eta=0.002,
                            nthreads=O.max_threads())
    Fe, ite, oke = OM.solve(*args, 0.2, start, tol=1e-10, max_iter=150, nthreads=O.max_threads())
    assert okr and oke
    assert np.abs(Fr - Fe).max() < 1e-4 * np.abs(Fe).max()


def test_ray_blended_quotient_at_mu_zero_approaches_the_vacuum_bc_solution():
    """Reading M8 at mu = 0 with the Ball-Chiu vertex (the paper's interaction, where the vacuum
    equation has the Nambu solution, A(0) = 1.18, M(0) = 0.30 GeV): the 2-D solve converges, and
    its distance to the pinned vacuum oracle's B(p^2) and the O(4) breaking |C - A| shrink as the
    grid is refined (observed: B 0.60 -> 0.070 -> 0.049 of max|B|, |C - A| 0.27 -> 0.17 ->
    0.056 on 12 x 8, 16 x 12, 24 x 16).  Without M8 this case runs away (one point's
    principal-value self-coupling exceeds 1)."""
    from paper_2012_03667_gb300 import inputs as I
    D_, om, m = 0.55, 0.678, 0.005
    A, B, it, ch, st = O.solve(O.Problem(n=128, n_theta=64, D=D_, omega=om, m=m), tol=1e-12,
                               nthreads=O.max_threads())
    assert st == 0
    sp, _, _, _ = O.radial_grid(128)
    errs = []
    for nr, n4 in ((12, 8), (16, 12)):
        w = I.mu_workload(n_r=nr, n_4=n4, n_z=16, n_mu=1, D=D_, omega=om, m=m)
        pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
        start = np.array([np.ones(len(w.p_abs))] * 3, dtype=np.complex128)
        F, it, ok = OM.solve(pa, p4a, w.q_abs, w.q4, *oracle_rule(w), D_, om, m, 0.0, start,
                             tol=1e-10, max_iter=100, ray_eta=0.002, nthreads=O.max_threads())
        assert ok
        s = w.p_abs ** 2 + w.p4 ** 2
        sel = (s > 1e-3) & (s < 10)
        Bv = np.interp(np.log(s[sel]), np.log(sp), B)
        errs.append((np.abs(F[2].real[sel] - Bv).max() / np.abs(Bv).max(),
                     np.abs(F[1] - F[0]).max()))
    assert errs[1][0] < errs[0][0] / 3 and errs[1][0] < 0.15
    assert errs[1][1] < 0.8 * errs[0][1]


def test_oracle_weights_are_gauss_rules_on_gauss_legendre_nodes():
    """The oracle's interpolatory weights, built from the nodes alone, integrate every monomial up
    to degree 2n - 1 exactly on Gauss-Legendre nodes (the Gauss property), so they are the Gauss
    weights; a rule with a wrong weight anywhere fails some degree."""
    for n in (8, 40, 64):
        t, _ = np.polynomial.legendre.leggauss(n)
        w = OM.interpolatory_weights(t)
        for k in range(2 * n):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert abs(float((w * t ** k).sum()) - exact) < 1e-13, (n, k)
    w = OM.interpolatory_weights(np.array([-0.5, 0.5]))  # two nodes, not Gauss: degree < 2 only
    assert np.allclose(w, [1.0, 1.0], rtol=0, atol=1e-15)


def test_oracle_measure_integrates_a_gaussian_in_closed_form():
    """Reading M5's measure |q|^2 d|q| dq_4 on the workload's product grid: the sum of
    exp(-(|q|^2 + q_4^2)/a) over the oracle's weights equals
    int_lo^hi x^2 e^{-x^2/a} dx * 2 int_lo^hi e^{-y^2/a} dy (q_4 on both sides of 0) in closed
    form with erf, to 1e-13 on the full 128 x 256 grid.  A dropped |q|^2, a missing mirror or a
    wrong Jacobian of the log map each miss it by orders of magnitude."""
    from math import erf, exp, pi, sqrt
    from paper_2012_03667_gb300 import inputs as I
    w = I.mu_workload(n_r=128, n_4=128, n_z=16, n_mu=1)
    a = 0.7
    QR, Q4 = np.meshgrid(w.q_abs, w.q4, indexing="ij")
    got = float((OM.measure(w.q_abs, w.q4, w.lo, w.hi) * np.exp(-(QR ** 2 + Q4 ** 2) / a).ravel())
                .sum())
    F = lambda x: a ** 1.5 * sqrt(pi) / 4 * erf(x / sqrt(a)) - a * x / 2 * exp(-x * x / a)
    G = lambda y: sqrt(pi * a) / 2 * erf(y / sqrt(a))
    exact = (F(w.hi) - F(w.lo)) * 2.0 * (G(w.hi) - G(w.lo))
    assert abs(got / exact - 1.0) < 1e-13
    # the angular rule: int_{-1}^{1} z^2 dz = 2/3
    wz = OM.angular_weights(w.z)
    assert abs(float((wz * w.z ** 2).sum()) - 2.0 / 3.0) < 1e-14
