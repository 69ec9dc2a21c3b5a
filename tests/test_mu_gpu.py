"""Finite chemical potential sweep on the GPU (include/qdse_mu.h) against the FP64 oracle.

The oracle (oracle/qdse_oracle_mu.cpp) sums every pair with explicit 4x4 complex Dirac matrices;
the CUDA path uses closed-form traces on a precomputed table of angular moments, drops pairs whose
Gaussian is below exp(-70) at every angle, and batches the chemical potentials in tiles.
Tolerances (relative to max |F - x0|, the self-energy part): FP64 1e-12; FP32 1e-4 on the small
grid and 5e-5 at full size (observed on the CPU with the same arithmetic: 2e-5 and 6e-6).
"""
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


pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def _iterates(w, qv, q4, mu_list, ext_idx=None):
    pv, p4 = (w.p_abs, w.p4) if ext_idx is None else (w.p_abs[ext_idx], w.p4[ext_idx])
    Fe = np.stack([I.mu_iterate(pv, p4, mu, w.m) for mu in mu_list])
    Fi = np.stack([I.mu_iterate(qv, q4, mu, w.m) for mu in mu_list])
    return Fe, Fi


def _gpu_sweep(QM, g, w, mu_list, Fe, Fi, vertex):
    dev = torch.device("cuda")
    Fe_t = torch.from_numpy(np.ascontiguousarray(Fe)).to(dev)
    Fi_t = torch.from_numpy(np.ascontiguousarray(Fi)).to(dev)
    out = torch.empty_like(Fe_t)
    g.sweep(mu_list, w.D, w.m, Fe_t, Fi_t, out, vertex=vertex)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _window_count(w):
    L = np.sqrt(70.0) * w.omega
    nr = np.array([(np.abs(w.q_abs - P) <= L).sum() for P in w.p_abs])
    nf = np.array([(np.abs(w.q4 - p4) <= L).sum() for p4 in w.p4])
    return int((nr * nf).sum())


SMALL = dict(n_r=20, n_4=12, n_z=32, n_mu=5)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (3, 1e-4)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("vertex", [0, 1], ids=["bc", "rl"])
def test_mu_sweep_matches_oracle(QM, precision, tol, vertex):
    """240 external x 480 internal points, 5 chemical potentials (a ragged tile for both tile
    widths) including mu = 0; pairs are dropped by the windows for |p| above 4 GeV."""
    w = I.mu_workload(**SMALL)
    mu_list = list(w.mu[:4]) + [0.0]
    qv, q4 = _internal(w)
    g = QM.MuGrid(w.p_abs, w.p4, w.q_abs, w.q4, *gpu_rule(w), w.omega, precision)
    assert g.info()["n_pairs"] == _window_count(w) < len(w.p_abs) * len(qv)
    Fe, Fi = _iterates(w, qv, q4, mu_list)
    got = _gpu_sweep(QM, g, w, mu_list, Fe, Fi, vertex)
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b, mu in enumerate(mu_list):
        ref = np.array(OM.sweep(w.p_abs, w.p4, qv, q4, *oracle_rule(w), w.D, w.omega, w.m, mu,
                                *Fe[b], *Fi[b], vertex=vertex, nthreads=0))
        scale = np.abs(ref - x0).max(axis=1)
        err = (np.abs(got[b] - ref).max(axis=1) / scale).max()
        assert err < tol, (b, mu, err)


def test_mu_batch_position_does_not_change_results(QM):
    """A mu gives bitwise the same output alone and in a later tile of a larger batch at the same
    slot of the tile (8 chemical potentials per warp in FP32): tiles, workspace growth and reuse
    do not change the arithmetic.  n_mu = 0 is a no-op."""
    w = I.mu_workload(**SMALL)
    qv, q4 = _internal(w)
    g = QM.MuGrid(w.p_abs, w.p4, w.q_abs, w.q4, *gpu_rule(w), w.omega, 3)
    first = list(w.mu[:5]) + [0.37, 0.02, 0.3]
    mu_big = first + first + first[:3]
    Fe, Fi = _iterates(w, qv, q4, mu_big)
    big = _gpu_sweep(QM, g, w, mu_big, Fe, Fi, 0)
    small = _gpu_sweep(QM, g, w, mu_big[:1], Fe[:1], Fi[:1], 0)
    assert np.array_equal(small[0], big[0])
    for b in range(8):
        assert np.array_equal(big[b], big[b + 8])
    for b in range(3):
        assert np.array_equal(big[b], big[b + 16])
    empty = torch.empty((0, 3, len(w.p_abs)), dtype=torch.complex128, device="cuda")
    g.sweep([], w.D, w.m, empty, torch.empty((0, 3, len(qv)), dtype=torch.complex128,
                                             device="cuda"), empty)


@pytest.mark.parametrize("precision,tol", [(3, 5e-5)], ids=["fp32"])
def test_mu_full_size_sampled_against_oracle(QM, precision, tol):
    """The full workload (16384 external x 32768 internal points, 64 angles, 256 chemical
    potentials) in one batched sweep; every output finite, and 6 sampled external points at 3
    chemical potentials (the largest, the smallest and one between) against the oracle."""
    w = I.mu_workload()
    qv, q4 = _internal(w)
    g = QM.MuGrid(w.p_abs, w.p4, w.q_abs, w.q4, *gpu_rule(w), w.omega, precision)
    assert g.info()["n_pairs"] == _window_count(w)
    Fe, Fi = _iterates(w, qv, q4, w.mu)
    got = _gpu_sweep(QM, g, w, list(w.mu), Fe, Fi, 0)
    assert np.isfinite(got).all()
    idx = np.array([0, 130, 1000, 5000, 9999, 16383])
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b in (int(np.argmax(w.mu)), int(np.argmin(w.mu)), 7):
        ref = np.array(OM.sweep(w.p_abs[idx], w.p4[idx], qv, q4, *oracle_rule(w), w.D,
                                w.omega, w.m, w.mu[b], *Fe[b][:, idx], *Fi[b], nthreads=0))
        scale = np.abs(ref - x0).max(axis=1)
        err = (np.abs(got[b][:, idx] - ref).max(axis=1) / scale).max()
        assert err < tol, (b, err)


# ---- the solve (interpolation + successive approximation) --------------------------------------
SOLVE = dict(n_r=12, n_4=8, n_z=24, n_mu=3)


def _solve_setup(QM, precision, D=None):
    w = I.mu_workload(**SOLVE)
    pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
    g = QM.MuGrid(pa, p4a, w.q_abs, w.q4, *gpu_rule(w), w.omega, precision, product=True)
    start = np.array([np.ones(len(w.p_abs)), np.ones(len(w.p_abs)),
                      0.3 * np.ones(len(w.p_abs))], dtype=np.complex128)
    return w, pa, p4a, g, start


def _oracle_solve(w, pa, p4a, D, mu, start, **kw):
    return OM.solve(pa, p4a, w.q_abs, w.q4, *oracle_rule(w), D, w.omega, w.m, mu, start, **kw)


def test_mu_solve_reaches_the_oracle_fixed_point_rainbow(QM):
    """FP64 solve of three chemical potentials at once (rainbow vertex, D = 0.93) against the
    oracle's solve: same fixed point to 1e-10 of max |F - x0|, same sweep count within one."""
    w, pa, p4a, g, start = _solve_setup(QM, 0)
    mu_list = [0.0, 0.1, 0.3]
    F = torch.from_numpy(np.stack([start] * 3)).cuda()
    iters, status = g.solve(mu_list, w.D, w.m, F, tol=1e-12, max_iter=200, vertex=1)
    assert list(status) == [0, 0, 0]
    got = F.cpu().numpy()
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b, mu in enumerate(mu_list):
        ref, it, ok = _oracle_solve(w, pa, p4a, w.D, mu, start, tol=1e-12, max_iter=200,
                                    vertex=OM.RL)
        assert ok and abs(int(iters[b]) - it) <= 1
        err = (np.abs(got[b] - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max()
        assert err < 1e-10, (mu, err)


@pytest.mark.parametrize("alpha", [1.0, 0.6])
def test_mu_solve_iterates_match_the_oracle_bc(QM, alpha):
    """Ball-Chiu vertex (D = 0.5, where the iteration contracts), exactly 15 sweeps (tol = 0) of
    two chemical potentials, damped and undamped: every element against the oracle to 1e-11."""
    w, pa, p4a, g, start = _solve_setup(QM, 0)
    D = 0.5
    mu_list = [0.05, 0.25]
    F = torch.from_numpy(np.stack([start] * 2)).cuda()
    iters, status = g.solve(mu_list, D, w.m, F, alpha=alpha, tol=0.0, max_iter=15, vertex=0)
    assert list(status) == [QM.Q.QDSE_ERR_NOT_CONVERGED] * 2 and list(iters) == [15, 15]
    got = F.cpu().numpy()
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b, mu in enumerate(mu_list):
        ref, _, _ = _oracle_solve(w, pa, p4a, D, mu, start, tol=0.0, max_iter=15, vertex=OM.BC,
                                  alpha=alpha)
        err = (np.abs(got[b] - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max()
        assert err < 1e-11, (mu, err)


def test_mu_mixed_solve_reaches_the_fp64_fixed_point(QM):
    """FP32 sweeps to a change of 1e-5, then FP64 sweeps on a grid of the same points to 1e-12:
    the result is the FP64 solve's fixed point to 1e-9."""
    w, pa, p4a, g64, start = _solve_setup(QM, 0)
    g32 = QM.MuGrid(pa, p4a, w.q_abs, w.q4, *gpu_rule(w), w.omega, 3, product=True)
    mu_list = [0.1, 0.3]
    F64 = torch.from_numpy(np.stack([start] * 2)).cuda()
    it64, st64 = g64.solve(mu_list, 0.5, w.m, F64, tol=1e-12, max_iter=400, vertex=0)
    Fm = torch.from_numpy(np.stack([start] * 2)).cuda()
    itm, stm = g32.solve(mu_list, 0.5, w.m, Fm, tol=1e-12, max_iter=400, vertex=0, refine=g64,
                         switch_tol=1e-5)
    assert list(st64) == [0, 0] and list(stm) == [0, 0]
    a, b = F64.cpu().numpy(), Fm.cpu().numpy()
    x0 = np.array([1.0, 1.0, w.m])[None, :, None]
    assert (np.abs(a - b).max(axis=2) / np.abs(a - x0).max(axis=2)).max() < 1e-9


def test_mu_solve_reports_non_convergence_and_non_finite_values(QM):
    """A start holding NaN at one chemical potential gives QDSE_ERR_NONFINITE there and leaves the
    other one unaffected; a sweep budget too small gives QDSE_ERR_NOT_CONVERGED; a grid made
    without the product form is refused."""
    w, pa, p4a, g, start = _solve_setup(QM, 0)
    bad = start.copy()
    bad[0, 3] = np.nan
    F = torch.from_numpy(np.stack([start, bad])).cuda()
    iters, status = g.solve([0.1, 0.1], w.D, w.m, F, tol=1e-12, max_iter=200, vertex=1)
    assert list(status) == [0, QM.Q.QDSE_ERR_NONFINITE]
    assert np.isfinite(F[0].cpu().numpy()).all()
    F = torch.from_numpy(np.stack([start])).cuda()
    iters, status = g.solve([0.1], w.D, w.m, F, tol=1e-12, max_iter=3, vertex=1)
    assert list(status) == [QM.Q.QDSE_ERR_NOT_CONVERGED] and list(iters) == [3]
    flat = QM.MuGrid(w.p_abs, w.p4, w.q_abs, w.q4, *gpu_rule(w), w.omega, 0)
    with pytest.raises(QM.Q.QdseError):
        flat.solve([0.1], w.D, w.m, F)


def _ray_setup(QM, precision):
    """The paper's interaction (D = 0.55, omega = 0.678) on the 12 x 8 product grid with 16 cosine
    nodes: the case where the exact quotient runs away at mu = 0 (reading M8's oracle pin)."""
    w = I.mu_workload(n_r=12, n_4=8, n_z=16, n_mu=1, D=0.55, omega=0.678)
    pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
    g = QM.MuGrid(pa, p4a, w.q_abs, w.q4, *gpu_rule(w), w.omega, precision, product=True)
    g.set_ray_quotient(0.002)
    start = np.array([np.ones(len(w.p_abs))] * 3, dtype=np.complex128)
    return w, pa, p4a, g, start


def test_mu_ray_quotient_iterates_match_the_oracle(QM):
    """Reading M8 on the GPU (eta = 0.002 GeV^2): exactly 12 sweeps of four chemical potentials,
    from mu = 0 (beta = 1 on every pair) through mu = 0.2 (the blend gone from most pairs), every
    element against the oracle's solve(ray_eta=0.002) to 1e-11 of max |F - x0|."""
    w, pa, p4a, g, start = _ray_setup(QM, 0)
    mu_list = [0.0, 0.01, 0.05, 0.2]
    F = torch.from_numpy(np.stack([start] * len(mu_list))).cuda()
    iters, status = g.solve(mu_list, 0.55, w.m, F, tol=0.0, max_iter=12, vertex=0)
    assert list(iters) == [12] * len(mu_list)
    got = F.cpu().numpy()
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b, mu in enumerate(mu_list):
        ref, _, _ = OM.solve(pa, p4a, w.q_abs, w.q4, *oracle_rule(w), 0.55, 0.678, w.m, mu,
                             start, tol=0.0, max_iter=12, ray_eta=0.002)
        err = (np.abs(got[b] - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max()
        assert err < 1e-11, (mu, err)


def test_mu_ray_quotient_converges_at_mu_zero_like_the_oracle(QM):
    """With reading M8 the mu = 0 solve converges (the exact quotient runs away there): the GPU's
    FP64 fixed point equals the oracle's to 1e-10 with the same sweep count within one, and the
    mixed solve (FP32 sweeps to 1e-5, then FP64) reaches the same point to 1e-9."""
    w, pa, p4a, g, start = _ray_setup(QM, 0)
    F = torch.from_numpy(np.stack([start])).cuda()
    iters, status = g.solve([0.0], 0.55, w.m, F, tol=1e-10, max_iter=80, vertex=0)
    ref, it, ok = OM.solve(pa, p4a, w.q_abs, w.q4, *oracle_rule(w), 0.55, 0.678, w.m, 0.0, start,
                           tol=1e-10, max_iter=80, ray_eta=0.002)
    assert ok and list(status) == [0] and abs(int(iters[0]) - it) <= 1
    got = F.cpu().numpy()[0]
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    assert (np.abs(got - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max() < 1e-10
    _, _, _, g32, _ = _ray_setup(QM, 3)
    Fm = torch.from_numpy(np.stack([start])).cuda()
    itm, stm = g32.solve([0.0], 0.55, w.m, Fm, tol=1e-10, max_iter=200, vertex=0, refine=g,
                         switch_tol=1e-5)
    assert list(stm) == [0]
    gm = Fm.cpu().numpy()[0]
    assert (np.abs(gm - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max() < 1e-9


def test_mu_ray_quotient_off_is_the_plain_sweep_and_bad_settings_are_refused(QM):
    """eta = 0 restores the exact quotient bitwise; a negative or non-finite eta and a grid made
    without the product form are refused."""
    w, pa, p4a, g, start = _ray_setup(QM, 0)
    plain = QM.MuGrid(pa, p4a, w.q_abs, w.q4, *gpu_rule(w), w.omega, 0, product=True)
    g.set_ray_quotient(0.0)
    F1 = torch.from_numpy(np.stack([start] * 2)).cuda()
    F2 = F1.clone()
    g.solve([0.1, 0.3], 0.55, w.m, F1, tol=0.0, max_iter=5, vertex=0)
    plain.solve([0.1, 0.3], 0.55, w.m, F2, tol=0.0, max_iter=5, vertex=0)
    assert torch.equal(F1, F2)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(QM.Q.QdseError):
            g.set_ray_quotient(bad)
    flat = QM.MuGrid(w.p_abs, w.p4, w.q_abs, w.q4, *gpu_rule(w), w.omega, 0)
    with pytest.raises(QM.Q.QdseError):
        flat.set_ray_quotient(0.002)


def test_mu_continuation_restarts_failed_mu_from_converged_neighbours(QM):
    """qdse_mu_solve_continued (rainbow vertex, FP64, 12 x 8 grid): the starts of mu = 0.1 and 0.2
    hold NaN, so the first solve ends QDSE_ERR_NONFINITE there.  The next round restarts 0.1 from
    0 and 0.2 from 0.3 (the nearest converged mu) and both converge, to the oracle's fixed point
    from the plain start to 1e-10; the two that converged at once are bitwise the plain solve's.
    max_rounds = 1 is qdse_mu_solve itself."""
    w, pa, p4a, g, start = _solve_setup(QM, 0)
    mu_list = [0.0, 0.1, 0.2, 0.3]
    bad = start.copy()
    bad[1, 5] = np.nan
    starts = np.stack([start, bad, bad, start])
    F = torch.from_numpy(starts).cuda()
    iters, status, rounds = g.solve_continued(mu_list, w.D, w.m, F, max_rounds=3, tol=1e-12,
                                              max_iter=200, vertex=1)
    assert list(status) == [0, 0, 0, 0] and list(rounds) == [0, 1, 1, 0]
    F1 = torch.from_numpy(starts).cuda()
    it1, st1 = g.solve(mu_list, w.D, w.m, F1, tol=1e-12, max_iter=200, vertex=1)
    assert list(st1) == [0, QM.Q.QDSE_ERR_NONFINITE, QM.Q.QDSE_ERR_NONFINITE, 0]
    assert torch.equal(F[0], F1[0]) and torch.equal(F[3], F1[3])
    assert iters[0] == it1[0] and iters[1] > it1[1]
    got = F.cpu().numpy()
    x0 = np.array([1.0, 1.0, w.m])[:, None]
    for b in (1, 2):
        ref, _, ok = _oracle_solve(w, pa, p4a, w.D, mu_list[b], start, tol=1e-12, max_iter=200,
                                   vertex=OM.RL)
        assert ok
        err = (np.abs(got[b] - ref).max(axis=1) / np.abs(ref - x0).max(axis=1)).max()
        assert err < 1e-10, (mu_list[b], err)
    F2 = torch.from_numpy(starts).cuda()
    it2, st2, r2 = g.solve_continued(mu_list, w.D, w.m, F2, max_rounds=1, tol=1e-12,
                                     max_iter=200, vertex=1)
    assert list(st2) == list(st1) and list(it2) == list(it1) and not r2.any()
    assert torch.equal(F2[0], F1[0]) and torch.equal(F2[3], F1[3])
