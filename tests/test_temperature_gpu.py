"""Finite temperature on the GPU (include/qdse_mu.h on a Matsubara grid) against the FP64 oracle.

Finite temperature (named as future work in the paper's Sec. V) is the finite-mu equation with the
fourth momentum on the fermion Matsubara frequencies (2n + 1) pi T and int dq_4/(2 pi) -> T sum_n
(readings T1, T2 of ``oracle_mu.matsubara_measure``, pinned in tests/test_oracle_temperature_pins.py).
The library needs no new kernel for it: the grid's internal q_4 are the frequencies, the external
p_4 axis is the positive ones, and the weights carry 2 pi T (formed on the package side by
``mu_rule.matsubara_weights``, independently of the oracle's).  Tolerances as for finite mu:
relative to max |F - x0|, FP64 1e-12 per sweep, 1e-10 at the fixed point, FP32 1e-4 per sweep.
"""
import numpy as np
import pytest

from oracle import oracle_mu as OM
from paper_2012_03667_gb300 import inputs as I
from paper_2012_03667_gb300 import mu_rule as MR

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ETA = 0.002  # reading M8's blend scale (GeV^2), as in the finite-mu solve workload


def gpu_rule(w):
    return MR.matsubara_weights(w.q_abs, w.q4, w.T, w.lo, w.hi), w.z, MR.angular_weights(w.z)


def oracle_rule(w):
    return OM.matsubara_measure(w.q_abs, w.q4, w.T, w.lo, w.hi), w.z, OM.angular_weights(w.z)


@pytest.fixture(scope="module")
def QM():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03667_gb300 import qdse_mu
    qdse_mu.load_library()
    return qdse_mu


def _internal(w):
    QR, Q4 = np.meshgrid(w.q_abs, w.q4, indexing="ij")
    return QR.ravel(), Q4.ravel()


def _start(n_ext, n_mu):
    s = np.zeros((n_mu, 3, n_ext), dtype=np.complex128)
    s[:, 0] = s[:, 1] = 1.0
    s[:, 2] = 0.3
    return s


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (3, 3e-4)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("vertex", [0, 1], ids=["bc", "rl"])
@pytest.mark.parametrize("T", [0.04, 0.25])
def test_matsubara_sweep_matches_oracle(QM, precision, tol, vertex, T):
    """One sweep on a 20 x 10-frequency grid (200 external x 400 internal points, 24 angles) for
    four chemical potentials including 0, from a smooth iterate, against the oracle's sweep with
    its own Matsubara measure.  The FP32 bound is 3e-4 rather than the finite-mu grid's 1e-4: at
    mu = 0 pairs of different frequencies can have |q|^2 + w_m^2 close to |p|^2 + w_n^2, and the
    Ball-Chiu quotients divide FP32 rounding of the numerator by that small difference (observed
    1.07e-4 at T = 0.04, mu = 0)."""
    w = I.matsubara_workload(T, n_r=20, n_4=10, n_z=24, n_mu=3)
    mu_list = list(w.mu) + [0.0]
    qv, q4 = _internal(w)
    g = QM.MuGrid(w.p_abs, w.p4, w.q_abs, w.q4, *gpu_rule(w), w.omega, precision)
    Fe = np.stack([I.mu_iterate(w.p_abs, w.p4, mu, w.m) for mu in mu_list])
    Fi = np.stack([I.mu_iterate(qv, q4, mu, w.m) for mu in mu_list])
    dev = torch.device("cuda")
    Fe_t, Fi_t = torch.from_numpy(Fe).to(dev), torch.from_numpy(Fi).to(dev)
    out = torch.empty_like(Fe_t)
    g.sweep(mu_list, w.D, w.m, Fe_t, Fi_t, out, vertex=vertex)
    got = out.cpu().numpy()
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b, mu in enumerate(mu_list):
        ref = np.array(OM.sweep(w.p_abs, w.p4, qv, q4, *oracle_rule(w), w.D, w.omega, w.m, mu,
                                *Fe[b], *Fi[b], vertex=vertex, nthreads=0))
        err = (np.abs(got[b] - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max()
        assert err < tol, (b, mu, err)


def _solve_setup(QM, T, precision):
    w = I.matsubara_workload(T, n_r=12, n_4=6, n_z=16, n_mu=1)
    pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
    g = QM.MuGrid(pa, p4a, w.q_abs, w.q4, *gpu_rule(w), w.omega, precision, product=True)
    g.set_ray_quotient(ETA)
    return w, pa, p4a, g


@pytest.mark.parametrize("T", [0.05, 0.2])
def test_matsubara_solve_reaches_the_oracle_fixed_point(QM, T):
    """Ball-Chiu solve at the paper's interaction (D = 0.55, omega = 0.678), mu = 0 and one mu > 0,
    with reading M8 on: the GPU's FP64 fixed point equals the oracle's to 1e-10 with the same sweep
    count within one; the mixed solve (FP32 sweeps to 1e-5, then FP64) reaches it to 1e-9.  At
    T = 0.05 the solution breaks chiral symmetry (M(0) near 0.48 GeV on this coarse grid), at
    T = 0.2 it is nearly restored (M(0) below 0.05 GeV): both branches are exercised.  (At T = 0.05
    the oracle does not converge at mu = 0.1 within 300 sweeps with eta = 0.002, the small-mu
    behaviour of the vacuum-like finite-mu solve, so that temperature takes mu = 0.2.)"""
    w, pa, p4a, g = _solve_setup(QM, T, 0)
    mu_list = [0.0, 0.2] if T < 0.1 else [0.0, 0.1]
    start = _start(len(w.p_abs), len(mu_list))
    F = torch.from_numpy(start.copy()).cuda()
    iters, status = g.solve(mu_list, w.D, w.m, F, tol=1e-10, max_iter=300, vertex=0)
    got = F.cpu().numpy()
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b, mu in enumerate(mu_list):
        ref, it, ok = OM.solve(pa, p4a, w.q_abs, w.q4, *oracle_rule(w), w.D, w.omega, w.m, mu,
                               start[b], tol=1e-10, max_iter=300, ray_eta=ETA)
        assert ok and status[b] == 0 and abs(int(iters[b]) - it) <= 1, (mu, it, iters[b])
        err = (np.abs(got[b] - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max()
        assert err < 1e-10, (mu, err)
    M0 = (got[0, 2, 0] / got[0, 0, 0]).real
    assert (M0 > 0.2) if T < 0.1 else (M0 < 0.1), M0
    _, _, _, g32 = _solve_setup(QM, T, 3)
    Fm = torch.from_numpy(start.copy()).cuda()
    itm, stm = g32.solve(mu_list, w.D, w.m, Fm, tol=1e-10, max_iter=400, vertex=0, refine=g,
                         switch_tol=1e-5)
    assert list(stm) == [0, 0]
    gm = Fm.cpu().numpy()
    assert (np.abs(gm - got).max(axis=2) / np.abs(got - x0[None]).max(axis=2)).max() < 1e-9
