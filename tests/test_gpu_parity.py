"""GPU parity: the CUDA path (through the C interface) against the FP64 oracle, element by element.

Tolerances: FP64 sweeps and FP64 maps/derivatives agree with the oracle to 1e-12 relative (only
summation order differs); converged FP64 solutions to 1e-10 (both sides iterate to 1e-13 or run the
same sweep count); the mixed-precision solve to 1e-8 (the target of the FP32 sweeps + FP64
refinement scheme).  Relative errors are max-norm over each function (max|dx| / max|x|).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2012_03667_gb300 import build as Bld
from paper_2012_03667_gb300 import inputs
from paper_2012_03667_gb300 import qdse as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    Bld.build()
    Q.load_library()
    torch.cuda.set_device(0)


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rel_pointwise(A, B, Ar, Br):
    """Reading R7's pointwise form: max relative error of A at every point and of B and M = B/A at
    the points where |B_i| >= 1e-6 max|B| (in the chiral limit B decays like exp(-p^2/w^2))."""
    e = float((np.abs(A - Ar) / np.abs(Ar)).max())
    keep = np.abs(Br) >= 1e-6 * np.abs(Br).max()
    if keep.any():
        e = max(e, float((np.abs(B - Br)[keep] / np.abs(Br)[keep]).max()),
                float((np.abs(B / A - Br / Ar)[keep] / np.abs(Br / Ar)[keep]).max()))
    return e


def problem(inst, mode=O.COLLOCATED, vertex=O.BC):
    return O.Problem(n=inst.n_p, n_theta=inst.n_theta, s_min=inst.s_min, s_max=inst.s_max,
                     grid_mode=mode, vertex=vertex, D=inst.D, omega=inst.omega, m=inst.m)


def grid(inst, mode=Q.QDSE_COLLOCATED):
    return Q.Grid(inst.n_p, inst.n_theta, inst.s_min, inst.s_max, mode)


def prm(inst):
    return [[inst.D, inst.omega, inst.m, 0.0]]


SMALL = inputs.SMALL
PAPER = inputs.PAPER
TINY = inputs.Instance(40, 24, 0.93, 0.5, 0.005)  # several 32-wide tiles + a ragged tail


# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [Q.QDSE_FP64, Q.QDSE_FP64_PRE])
@pytest.mark.parametrize("inst", [SMALL, PAPER, TINY], ids=["small", "paper", "tiny"])
def test_fp64_sweeps_match_oracle_iterate_by_iterate(precision, inst):
    ctx = Q.Context(grid(inst), 1, precision=precision)
    pr = problem(inst)
    A = dev(np.full(inst.n_p, 1.0)); B = dev(np.full(inst.n_p, 0.3))
    Ao, Bo = np.full(inst.n_p, 1.0), np.full(inst.n_p, 0.3)
    done = 0
    for n in (1, 2, 5):
        ctx.qdse_iterate(prm(inst), A, B, n - done)
        for _ in range(n - done):
            Ao, Bo = O.sweep(pr, Ao, Bo)
        done = n
        assert rel(host(A), Ao) < 1e-12, n
        assert rel(host(B), Bo) < 1e-12, n


@pytest.mark.parametrize("mode", [O.COLLOCATED, O.STAGGERED])
@pytest.mark.parametrize("vertex", [O.BC, O.RL])
def test_map_residual_matches_oracle_random_inputs(mode, vertex):
    inst = TINY
    rng = np.random.default_rng(3)
    A = 1 + rng.uniform(0, 1.5, inst.n_p); B = rng.uniform(0.01, 0.8, inst.n_p)
    Fo_A, Fo_B = O.sweep(problem(inst, mode, vertex), A, B)
    for precision in (Q.QDSE_FP64, Q.QDSE_FP64_PRE):
        ctx = Q.Context(grid(inst, mode), 1, precision=precision, vertex=vertex)
        FA = dev(np.zeros(inst.n_p)); FB = dev(np.zeros(inst.n_p)); r = dev(np.zeros(1))
        ctx.qdse_residual(prm(inst), dev(A), dev(B), FA, FB, r)
        assert rel(host(FA), Fo_A) < 1e-12
        assert rel(host(FB), Fo_B) < 1e-12


def test_fp32_sweeps_track_oracle():
    inst = SMALL
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_FP32)
    A = dev(np.full(inst.n_p, 1.0)); B = dev(np.full(inst.n_p, 0.3))
    ctx.qdse_iterate(prm(inst), A, B, 3)
    Ao, Bo = np.full(inst.n_p, 1.0), np.full(inst.n_p, 0.3)
    for _ in range(3):
        Ao, Bo = O.sweep(problem(inst), Ao, Bo)
    assert rel(host(A), Ao) < 2e-5 and rel(host(B), Bo) < 2e-5


RAGGED32 = [inputs.Instance(37, 16, 0.93, 0.5, 0.005), inputs.Instance(64, 32, 0.7, 0.45, 0.05),
            inputs.Instance(130, 24, 1.1, 0.6, 0.1), inputs.Instance(300, 32, 0.6, 0.4, 0.0)]


@pytest.mark.parametrize("kind", ["slab", "ring", "groups"])
def test_fp32_sweep_kernels_track_oracle_on_ragged_batch(kind, monkeypatch):
    """The FP32 sweep kernels (slabs of row groups and single row groups through the shared-memory
    ring, and the register-only row groups) on one ragged batch: last groups of 1, 2 and 4 rows,
    last slabs of 1 to 8 groups, bands from a few columns to a few hundred (tiles split at 128
    columns), three sweeps each against the oracle's FP64 sweeps."""
    monkeypatch.setenv("QDSE_SWEEP", kind)
    ctx = Q.Context([grid(i) for i in RAGGED32], precision=Q.QDSE_FP32)
    x_off = ctx.layout()
    A = dev(np.ones(ctx.n_total)); B = dev(np.full(ctx.n_total, 0.3))
    ctx.qdse_iterate([[i.D, i.omega, i.m, 0.0] for i in RAGGED32], A, B, 3)
    Ah, Bh = host(A), host(B)
    for b, inst in enumerate(RAGGED32):
        Ao, Bo = np.ones(inst.n_p), np.full(inst.n_p, 0.3)
        for _ in range(3):
            Ao, Bo = O.sweep(problem(inst), Ao, Bo)
        sl = slice(x_off[b], x_off[b + 1])
        assert rel(Ah[sl], Ao) < 2e-5 and rel(Bh[sl], Bo) < 2e-5, (kind, b)


def test_narrow_group_sweep_is_bitwise_the_ring_on_a_ragged_batch(monkeypatch):
    """The narrow-group kernel on the ragged batch (last groups of 1, 2 and 4 rows, odd sizes,
    bands from a few columns up): three FP32 sweeps bitwise equal to the ring sweep alone."""
    out = []
    for narrow in ("0", "1"):
        monkeypatch.setenv("QDSE_NARROW", narrow)
        ctx = Q.Context([grid(i) for i in RAGGED32], precision=Q.QDSE_FP32)
        A = dev(np.ones(ctx.n_total)); B = dev(np.full(ctx.n_total, 0.3))
        ctx.qdse_iterate([[i.D, i.omega, i.m, 0.0] for i in RAGGED32], A, B, 3)
        out.append((host(A), host(B)))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_jvp_matches_complex_step_jacobian():
    inst = TINY
    rng = np.random.default_rng(9)
    A = 1 + rng.uniform(0, 1.5, inst.n_p); B = rng.uniform(0.05, 0.8, inst.n_p)
    J = O.jacobian(problem(inst), A, B)
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_FP64_PRE)
    for trial in range(3):
        v = rng.normal(size=2 * inst.n_p)
        JA = dev(np.zeros(inst.n_p)); JB = dev(np.zeros(inst.n_p))
        ctx.qdse_jvp(prm(inst), dev(A), dev(B), dev(v[:inst.n_p]), dev(v[inst.n_p:]), JA, JB)
        ref = J @ v
        got = np.concatenate([host(JA), host(JB)])
        assert rel(got, ref) < 1e-11


@pytest.mark.parametrize("mode", [O.COLLOCATED, O.STAGGERED])
@pytest.mark.parametrize("vertex", [O.BC, O.RL])
def test_vjp_matches_transposed_jacobian(vertex, mode):
    inst = TINY
    rng = np.random.default_rng(4 + mode)
    A = 1 + rng.uniform(0, 1.5, inst.n_p); B = rng.uniform(0.05, 0.8, inst.n_p)
    J = O.jacobian(problem(inst, mode, vertex), A, B)
    ctx = Q.Context(grid(inst, mode), 1, precision=Q.QDSE_FP64_PRE, vertex=vertex)
    w = rng.normal(size=2 * inst.n_p)
    JA = dev(np.zeros(inst.n_p)); JB = dev(np.zeros(inst.n_p))
    ctx.qdse_vjp(prm(inst), dev(A), dev(B), dev(w[:inst.n_p]), dev(w[inst.n_p:]), JA, JB)
    got = np.concatenate([host(JA), host(JB)])
    assert rel(got, J.T @ w) < 1e-11


# ------------------------------------------------------------------------------------------------
def oracle_fixed_point(inst, mode=O.COLLOCATED, vertex=O.BC):
    A, B, it, ch, st = O.solve(problem(inst, mode, vertex), tol=1e-13, max_iter=20000,
                               nthreads=O.max_threads())
    assert st == 0
    return A, B, it


@pytest.mark.parametrize("precision,tol", [(Q.QDSE_FP64, 1e-10), (Q.QDSE_FP64_PRE, 1e-10),
                                           (Q.QDSE_MIXED, 1e-8)])
@pytest.mark.parametrize("inst", [SMALL, PAPER], ids=["small", "paper"])
def test_solve_matches_oracle_fixed_point(precision, tol, inst):
    Ar, Br, it = oracle_fixed_point(inst)
    ctx = Q.Context(grid(inst), 1, precision=precision, tol=1e-13, max_iter=40000)
    A = dev(np.full(inst.n_p, 1.0)); B = dev(np.full(inst.n_p, 0.3))
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_solve(prm(inst), A, B, iters, st)
    assert int(st.item()) == Q.QDSE_OK
    eA, eB = rel(host(A), Ar), rel(host(B), Br)
    eM = rel(host(B) / host(A), Br / Ar)
    assert max(eA, eB, eM) < tol, (eA, eB, eM)
    assert rel_pointwise(host(A), host(B), Ar, Br) < tol


def test_staggered_solve_matches_oracle():
    inst = PAPER
    Ar, Br, it = oracle_fixed_point(inst, O.STAGGERED)
    ctx = Q.Context(grid(inst, Q.QDSE_STAGGERED), 1, precision=Q.QDSE_MIXED, tol=1e-13)
    A = dev(np.full(inst.n_p, 1.0)); B = dev(np.full(inst.n_p, 0.3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_solve(prm(inst), A, B, None, st)
    assert int(st.item()) == 0
    assert rel(host(A), Ar) < 1e-8 and rel(host(B), Br) < 1e-8
    assert rel_pointwise(host(A), host(B), Ar, Br) < 1e-8


def test_ragged_batch_matches_per_instance_oracle():
    insts = [inputs.Instance(48, 16, 0.55, 0.678, 0.005), inputs.Instance(64, 24, 0.7, 0.6, 0.05),
             inputs.Instance(37, 8, 0.6, 0.55, 0.0), inputs.Instance(72, 32, 0.5, 0.7, 0.1)]
    grids = [grid(i) for i in insts]
    ctx = Q.Context(grids, precision=Q.QDSE_MIXED, tol=1e-13, max_iter=40000)
    x_off = ctx.layout()
    A = dev(np.ones(ctx.n_total)); B = dev(np.full(ctx.n_total, 0.3))
    st = torch.zeros(len(insts), dtype=torch.int32, device="cuda")
    ctx.qdse_solve([[i.D, i.omega, i.m, 0] for i in insts], A, B, None, st)
    Ah, Bh = host(A), host(B)
    assert np.all(host(st) == 0)
    for b, inst in enumerate(insts):
        Ar, Br, _ = oracle_fixed_point(inst)
        sl = slice(x_off[b], x_off[b + 1])
        assert rel(Ah[sl], Ar) < 1e-8 and rel(Bh[sl], Br) < 1e-8, b
        assert rel_pointwise(Ah[sl], Bh[sl], Ar, Br) < 1e-8, b


SCAN_SHAPES = [inputs.Instance(384, 32, 0.55, 0.678, 0.005), inputs.Instance(512, 64, 0.6, 0.55, 0.02),
               inputs.Instance(384, 64, 0.5, 0.6, 0.1), inputs.Instance(512, 32, 0.45, 0.7, 0.0)]


def test_mixed_solve_matches_oracle_at_the_scan_shapes():
    """The scan's large shapes (N_q = 384 and 512 with N_theta = 32 and 64) in one ragged batch, at
    interactions below the BC fold (D omega <= 0.37), including the chiral limit m = 0: the mixed
    solve against the oracle's fixed point to 1e-8, norm-relative and pointwise (R7)."""
    ctx = Q.Context([grid(i) for i in SCAN_SHAPES], precision=Q.QDSE_MIXED, tol=1e-13,
                    max_iter=40000)
    x_off = ctx.layout()
    A = dev(np.ones(ctx.n_total)); B = dev(np.full(ctx.n_total, 0.3))
    st = torch.zeros(len(SCAN_SHAPES), dtype=torch.int32, device="cuda")
    ctx.qdse_solve([[i.D, i.omega, i.m, 0] for i in SCAN_SHAPES], A, B, None, st)
    Ah, Bh = host(A), host(B)
    assert np.all(host(st) == 0)
    for b, inst in enumerate(SCAN_SHAPES):
        Ar, Br, _ = oracle_fixed_point(inst)
        sl = slice(x_off[b], x_off[b + 1])
        assert rel(Ah[sl], Ar) < 1e-8 and rel(Bh[sl], Br) < 1e-8, b
        assert rel(Bh[sl] / Ah[sl], Br / Ar) < 1e-8, b
        assert rel_pointwise(Ah[sl], Bh[sl], Ar, Br) < 1e-8, b


LARGE_PAPER = inputs.Instance(512, 128, 0.55, 0.678, 0.005)


@pytest.mark.parametrize("precision", [Q.QDSE_FP64, Q.QDSE_FP64_PRE])
def test_large_grid_first_sweeps_match_oracle(precision):
    """N = 512, N_theta = 128, D = 0.93, w = 0.5: sweep-by-sweep parity.  At these parameters the
    Picard iteration is chaotic (rounding differences grow ~10x per 10 sweeps after the first
    ~20), so iterates are compared while the two trajectories are still the same trajectory."""
    inst = inputs.LARGE
    pr = problem(inst)
    ctx = Q.Context(grid(inst), 1, precision=precision)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    Ao, Bo = np.ones(inst.n_p), np.full(inst.n_p, 0.3)
    done = 0
    for n, tol in ((1, 1e-13), (5, 1e-12), (15, 1e-11)):
        ctx.qdse_iterate(prm(inst), A, B, n - done)
        for _ in range(n - done):
            Ao, Bo = O.sweep(pr, Ao, Bo, nthreads=O.max_threads())
        done = n
        assert rel(host(A), Ao) < tol and rel(host(B), Bo) < tol, n


def test_large_grid_solution_is_a_fixed_point_of_the_oracle_map():
    """The FP64 GPU solve at N = 512, N_theta = 128, D = 0.93 (deterministic on the GPU) ends on a
    fixed point of the oracle's map, checked on every row."""
    inst = inputs.LARGE
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_FP64, tol=1e-11, max_iter=6000)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_solve(prm(inst), A, B, None, st)
    assert int(st.item()) == 0
    Ah, Bh = host(A), host(B)
    Fa, Fb = O.sweep(problem(inst), Ah, Bh, nthreads=O.max_threads())
    assert rel(Fa, Ah) < 1e-9 and rel(Fb, Bh) < 1e-9


@pytest.mark.parametrize("precision,tol", [(Q.QDSE_FP64_PRE, 1e-10), (Q.QDSE_MIXED, 1e-8)])
def test_large_grid_solve_matches_oracle_paper_parameters(precision, tol):
    """N = 512, N_theta = 128 with the paper's D = 0.55, w = 0.678 (a unique attracting fixed
    point): GPU solution against the oracle's, element by element."""
    inst = LARGE_PAPER
    Ar, Br, _ = oracle_fixed_point(inst)
    ctx = Q.Context(grid(inst), 1, precision=precision, tol=1e-13, max_iter=5000)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_solve(prm(inst), A, B, None, st)
    assert int(st.item()) == 0
    assert rel(host(A), Ar) < tol and rel(host(B), Br) < tol
    assert rel(host(B) / host(A), Br / Ar) < tol


def test_mixed_solution_is_an_fp64_fixed_point_in_the_chaotic_regime():
    """D = 0.93 on the large grid: whichever fixed point the mixed-precision solve reaches, it is
    an FP64 fixed point to 1e-8: plain FP64 successive approximation restarted from it stays put,
    and the oracle's map leaves it unchanged."""
    inst = inputs.LARGE
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_MIXED, tol=1e-11, max_iter=6000)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_solve(prm(inst), A, B, None, st)
    s = int(st.item())
    assert s in (Q.QDSE_OK, Q.QDSE_ERR_NOT_CONVERGED, Q.QDSE_ERR_NONFINITE)
    if s != Q.QDSE_OK:
        # Picard is chaotic here: a trajectory can end in a cycle or leave through NaN, and
        # which one depends on rounding order; only a reached fixed point can be checked
        pytest.skip("the mixed trajectory ended in a cycle or diverged (no fixed point reached)")
    Ah, Bh = host(A), host(B)
    Fa, Fb = O.sweep(problem(inst), Ah, Bh, nthreads=O.max_threads())
    assert rel(Fa, Ah) < 1e-9 and rel(Fb, Bh) < 1e-9
    c64 = Q.Context(grid(inst), 1, precision=Q.QDSE_FP64, tol=1e-10, max_iter=2000)
    A2, B2 = A.clone(), B.clone()
    c64.qdse_solve(prm(inst), A2, B2, None, st)
    assert int(st.item()) == 0
    assert rel(host(A2), Ah) < 1e-8 and rel(host(B2), Bh) < 1e-8


# ------------------------------------------------------------------------------------------------
def test_adjoint_matches_oracle_adjoint():
    inst = inputs.Instance(32, 16, 0.55, 0.678, 0.02)
    pr = problem(inst)
    Ar, Br, it, ch, st = O.solve(pr, tol=1e-14, max_iter=20000)
    rng = np.random.default_rng(1)
    gA = rng.normal(size=inst.n_p); gB = rng.normal(size=inst.n_p)
    gp_ref, lam_ref = O.adjoint(pr, Ar, Br, gA, gB)
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_MIXED, tol=1e-14, max_iter=40000)
    gp = dev(np.zeros(4)); lam = dev(np.zeros(2 * inst.n_p))
    ist = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_adjoint(prm(inst), dev(Ar), dev(Br), dev(gA), dev(gB), gp, lam, ist)
    assert int(ist.item()) == 0
    assert rel(host(lam), lam_ref) < 1e-10
    got = host(gp)
    np.testing.assert_allclose(got[:3], gp_ref[:3], rtol=1e-9)
    assert got[3] == 0.0


@pytest.mark.parametrize("inst", [inputs.Instance(256, 64, 0.55, 0.678, 0.02),
                                  inputs.Instance(256, 64, 0.6, 0.55, 0.08)], ids=["paper", "scan"])
def test_adjoint_matches_oracle_adjoint_at_the_adjoint_workload_shape(inst):
    """N_q = 256, N_theta = 64 (the shape of the 1024-instance adjoint workload): lambda and the
    parameter gradients of the GPU adjoint against the oracle's dense-LU adjoint."""
    pr = problem(inst)
    Ar, Br, it, ch, st = O.solve(pr, tol=1e-14, max_iter=20000, nthreads=O.max_threads())
    assert st == 0
    rng = np.random.default_rng(inst.n_p + int(100 * inst.D))
    gA = rng.normal(size=inst.n_p); gB = rng.normal(size=inst.n_p)
    gp_ref, lam_ref = O.adjoint(pr, Ar, Br, gA, gB, nthreads=O.max_threads())
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_MIXED, tol=1e-14, max_iter=40000)
    gp = dev(np.zeros(4)); lam = dev(np.zeros(2 * inst.n_p))
    ist = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_adjoint(prm(inst), dev(Ar), dev(Br), dev(gA), dev(gB), gp, lam, ist)
    assert int(ist.item()) == 0
    assert rel(host(lam), lam_ref) < 1e-9
    got = host(gp)
    np.testing.assert_allclose(got[:3], gp_ref[:3], rtol=1e-8)
    assert got[3] == 0.0


def test_mixed_precision_adjoint_matches_the_fp64_adjoint_with_few_fp64_sweeps():
    """The MIXED context's adjoint (FP32 inner transposed sweeps, FP64 residuals of
    lambda = J^T lambda + g) against the FP64_PRE context's plain FP64 successive approximation,
    on a small batch at the adjoint workload's shape: the same lambda and parameter gradients to
    1e-10, every instance converged, and far fewer FP64 sweeps (the FP32 ones do the iterating)."""
    batch = [inputs.Instance(256, 64, D, om, m) for D, om, m in
             ((0.55, 0.678, 0.02), (0.6, 0.55, 0.08), (0.55, 0.6, 0.05), (0.5, 0.6, 0.1))]
    grids = [grid(b) for b in batch]
    prms = [[b.D, b.omega, b.m, 0.0] for b in batch]
    fwd = Q.Context(grids, precision=Q.QDSE_FP64_PRE, tol=1e-14, max_iter=40000)
    A = dev(np.ones(fwd.n_total)); B = dev(np.full(fwd.n_total, 0.3))
    st = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
    fwd.qdse_solve(prms, A, B, None, st)
    assert np.all(host(st) == 0)
    rng = np.random.default_rng(11)
    gA = dev(rng.normal(size=fwd.n_total)); gB = dev(rng.normal(size=fwd.n_total))
    out = {}
    for precision in (Q.QDSE_FP64_PRE, Q.QDSE_MIXED):
        ctx = Q.Context(grids, precision=precision, tol=1e-13, max_iter=40000)
        gp = dev(np.zeros(4 * len(batch))); lam = dev(np.zeros(2 * ctx.n_total))
        ist = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
        ctx.qdse_adjoint(prms, A, B, gA, gB, gp, lam, ist)
        assert np.all(host(ist) == 0), precision
        out[precision] = (host(lam), host(gp), ctx.qdse_last_stats())
    (l64, g64, s64), (lmx, gmx, smx) = out[Q.QDSE_FP64_PRE], out[Q.QDSE_MIXED]
    assert rel(lmx, l64) < 1e-10
    np.testing.assert_allclose(gmx.reshape(-1, 4)[:, :3], g64.reshape(-1, 4)[:, :3], rtol=1e-9)
    assert smx["fp64_sweeps"] * 5 < s64["fp64_sweeps"], (smx, s64)
    assert smx["fp32_sweeps"] > 0


def test_adjoint_on_a_staggered_grid_matches_oracle_adjoint():
    """The paper's own grid mode (Eqs. pqrelationship, chazhiresult): the transposed fixed point and
    the parameter gradients against the oracle's dense-LU adjoint of the staggered sweep."""
    inst = inputs.Instance(40, 16, 0.55, 0.678, 0.02)
    pr = problem(inst, O.STAGGERED)
    Ar, Br, it, ch, st = O.solve(pr, tol=1e-14, max_iter=20000)
    assert st == 0
    rng = np.random.default_rng(6)
    gA = rng.normal(size=inst.n_p); gB = rng.normal(size=inst.n_p)
    gp_ref, lam_ref = O.adjoint(pr, Ar, Br, gA, gB)
    ctx = Q.Context(grid(inst, Q.QDSE_STAGGERED), 1, precision=Q.QDSE_MIXED, tol=1e-14,
                    max_iter=40000)
    gp = dev(np.zeros(4)); lam = dev(np.zeros(2 * inst.n_p))
    ist = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_adjoint(prm(inst), dev(Ar), dev(Br), dev(gA), dev(gB), gp, lam, ist)
    assert int(ist.item()) == 0
    assert rel(host(lam), lam_ref) < 1e-10
    got = host(gp)
    np.testing.assert_allclose(got[:3], gp_ref[:3], rtol=1e-9)


def test_condensate_and_its_cotangent():
    inst = PAPER
    Ar, Br, _ = oracle_fixed_point(inst)
    ctx = Q.Context(grid(inst), 1)
    out = dev(np.zeros(1))
    ctx.qdse_condensate(dev(Ar), dev(Br), out)
    ref = O.condensate(problem(inst), Ar, Br)
    assert host(out)[0] == pytest.approx(ref, rel=1e-13)
    gA = dev(np.zeros(inst.n_p)); gB = dev(np.zeros(inst.n_p))
    ctx.qdse_condensate_vjp(dev(Ar), dev(Br), dev([1.0]), gA, gB)
    h = 1e-6
    for arr, g in ((Ar, gA), (Br, gB)):
        gh = host(g)
        scale = np.abs(gh).max()
        for k in (0, 20, 30, 40, 50):
            xp = arr.copy(); xp[k] += h; xm = arr.copy(); xm[k] -= h
            a1 = (xp, Br) if arr is Ar else (Ar, xp)
            a2 = (xm, Br) if arr is Ar else (Ar, xm)
            fd = (O.condensate(problem(inst), *a1) - O.condensate(problem(inst), *a2)) / (2 * h)
            # central differences carry ~1e-16/h rounding: compare on the gradient's own scale
            assert abs(gh[k] - fd) < 1e-6 * scale, (k, gh[k], fd)


# ------------------------------------------------------------------------------------------------
def test_status_not_converged_nonfinite_and_timeout():
    inst = SMALL
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_MIXED, max_iter=1)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    it = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.qdse_solve(prm(inst), A, B, it, st)
    assert int(st.item()) == Q.QDSE_ERR_NOT_CONVERGED and int(it.item()) == 1
    # a NaN in the start is reported per instance
    ctx.set_options(max_iter=100)
    a = np.ones(inst.n_p); a[10] = np.nan
    A = dev(a); B = dev(np.full(inst.n_p, 0.3))
    ctx.qdse_solve(prm(inst), A, B, None, st)
    assert int(st.item()) == Q.QDSE_ERR_NONFINITE
    # a wall-clock limit that runs out ends the call with QDSE_ERR_TIMEOUT (host-side check)
    ctx3 = Q.Context(grid(inst), 1, precision=Q.QDSE_FP64, max_iter=10 ** 6, time_limit=1e-9,
                     tol=0.0)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    with pytest.raises(Q.QdseError) as e:
        ctx3.qdse_solve(prm(inst), A, B, None, st)
    assert e.value.status == Q.QDSE_ERR_TIMEOUT
    assert int(st.item()) == Q.QDSE_ERR_TIMEOUT


def test_bounded_sweep_wait_runs_out_and_reports_timeout(monkeypatch):
    """The sweep's waits are bounded: with the test switch QDSE_TEST_STALL=1 every tile expects
    16 bytes more than its copies deliver, so each wait runs out after its clock budget (about a
    second).  The kernel flags it and returns, later launches of the solve stop at once, the call
    returns QDSE_ERR_TIMEOUT with per-instance TIMEOUT status, and the GPU stays usable: a fresh
    context then solves normally."""
    monkeypatch.delenv("QDSE_SWEEP", raising=False)
    monkeypatch.setenv("QDSE_TEST_STALL", "1")
    inst = PAPER
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_MIXED)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(Q.QdseError) as e:
        ctx.qdse_solve(prm(inst), A, B, None, st)
    assert e.value.status == Q.QDSE_ERR_TIMEOUT
    assert int(st.item()) == Q.QDSE_ERR_TIMEOUT
    ctx.close()
    monkeypatch.delenv("QDSE_TEST_STALL")
    ctx2 = Q.Context(grid(inst), 1, precision=Q.QDSE_MIXED, tol=1e-13, max_iter=40000)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    ctx2.qdse_solve(prm(inst), A, B, None, st)
    assert int(st.item()) == Q.QDSE_OK
    Ar, Br, _ = oracle_fixed_point(inst)
    assert rel(host(A), Ar) < 1e-8 and rel(host(B), Br) < 1e-8


def test_bad_parameters_rejected():
    ctx = Q.Context(grid(SMALL), 1)
    A = dev(np.ones(SMALL.n_p)); B = dev(np.full(SMALL.n_p, 0.3))
    for p in ([[0.93, -0.5, 0.005, 0]], [[np.nan, 0.5, 0.005, 0]], [[0.93, 0.5, np.inf, 0]]):
        with pytest.raises(Q.QdseError) as e:
            ctx.qdse_solve(p, A, B)
        assert e.value.status == Q.QDSE_ERR_ARG
    with pytest.raises(Q.QdseError) as e:
        ctx.qdse_solve([[0.93, 0.5, 0.005, 0.1]], A, B)
    assert e.value.status == Q.QDSE_ERR_UNSUPPORTED


def test_chiral_limit_keeps_b_zero():
    inst = inputs.Instance(48, 16, 0.55, 0.678, 0.0)
    for precision in (Q.QDSE_FP64, Q.QDSE_MIXED):
        ctx = Q.Context(grid(inst), 1, precision=precision, tol=1e-12)
        A = dev(np.ones(inst.n_p)); B = dev(np.zeros(inst.n_p))
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        ctx.qdse_solve(prm(inst), A, B, None, st)
        assert int(st.item()) == 0
        assert np.all(host(B) == 0.0)


def test_minimum_sizes():
    inst = inputs.Instance(3, 1, 0.55, 0.678, 0.005, 1e-2, 1e2)
    pr = problem(inst)
    Ao, Bo = O.sweep(pr, np.ones(3), np.full(3, 0.3))
    for precision in (Q.QDSE_FP64, Q.QDSE_FP64_PRE):
        ctx = Q.Context(grid(inst), 1, precision=precision)
        A = dev(np.ones(3)); B = dev(np.full(3, 0.3))
        ctx.qdse_iterate(prm(inst), A, B, 1)
        assert rel(host(A), Ao) < 1e-12 and rel(host(B), Bo) < 1e-12


def test_host_buffer_entry_point_equals_device_path():
    inst = PAPER
    ctx = Q.Context(grid(inst), 1, precision=Q.QDSE_MIXED, tol=1e-12)
    A = dev(np.ones(inst.n_p)); B = dev(np.full(inst.n_p, 0.3))
    ctx.qdse_solve(prm(inst), A, B)
    Ah = np.ones(inst.n_p); Bh = np.full(inst.n_p, 0.3)
    it = np.zeros(1, dtype=np.int32); st = np.zeros(1, dtype=np.int32)
    ctx.qdse_solve_host(prm(inst), Ah, Bh, it, st)
    assert st[0] == 0 and it[0] > 0
    np.testing.assert_array_equal(Ah, host(A))
    np.testing.assert_array_equal(Bh, host(B))


def test_autograd_chiral_susceptibility_matches_finite_differences():
    """torch.autograd through the solve (implicit adjoint) and the condensate: dC/dm, dC/dD,
    dC/dw against central differences of converged solves (h = 1e-5)."""
    from paper_2012_03667_gb300 import autograd as AG
    insts = [inputs.Instance(48, 24, 0.55, 0.678, 0.02), inputs.Instance(40, 16, 0.6, 0.6, 0.05)]
    ctx = Q.Context([grid(i) for i in insts], precision=Q.QDSE_MIXED, tol=1e-14, max_iter=40000)
    theta = torch.tensor([[i.m, i.D, i.omega] for i in insts], dtype=torch.float64,
                         requires_grad=True)
    A, B = AG.gap_solve(ctx, theta)
    C = AG.condensate(ctx, A, B)
    C.sum().backward()
    g = theta.grad.numpy()
    h = 1e-5
    for b, inst in enumerate(insts):
        for t, key in enumerate(("m", "D", "omega")):
            vals = []
            for sgn in (1, -1):
                kw = dict(inst.__dict__)
                kw[key] += sgn * h
                Ar, Br, _ = oracle_fixed_point(inputs.Instance(**kw))
                vals.append(O.condensate(problem(inputs.Instance(**kw)), Ar, Br))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert g[b, t] == pytest.approx(fd, rel=2e-5, abs=1e-9), (b, key, g[b, t], fd)
