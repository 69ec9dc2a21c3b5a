"""GPU tests of the batched solver's own machinery (beyond parity with the oracle): the cycle stop
on the full 4096-instance scan, and the FP32-pipe kernel precompute against the FP64 one."""
import numpy as np
import pytest
import torch

from paper_2012_03667_gb300 import build as Bld
from paper_2012_03667_gb300 import inputs
from paper_2012_03667_gb300 import qdse as Q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    Bld.build()
    Q.load_library()
    torch.cuda.set_device(0)


def _solve_scan(batch, stop_cycles, max_iter=5000, stall_window=0):
    grids = [Q.Grid(b.n_p, b.n_theta, b.s_min, b.s_max) for b in batch]
    ctx = Q.Context(grids, precision=Q.QDSE_MIXED, tol=1e-10, max_iter=max_iter,
                    stop_cycles=stop_cycles, stall_window=stall_window)
    n = ctx.n_total
    A = torch.ones(n, dtype=torch.float64, device="cuda")
    B = torch.full((n,), 0.3, dtype=torch.float64, device="cuda")
    st = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
    it = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
    ctx.qdse_solve([[b.D, b.omega, b.m, 0.0] for b in batch], A, B, it, st)
    out = (A.cpu().numpy(), B.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(),
           ctx.qdse_last_instance_stats(), ctx.layout())
    ctx.close()
    return out


def test_cycle_stop_leaves_the_converged_set_of_the_scan_unchanged():
    """The 4096-instance scan at the same cap (5000 sweeps) with and without the cycle stop: the
    same instances converge, to bitwise the same A and B, with the same sweep counts; every
    instance the stop ended reports a cycle period and ended before the cap as NOT_CONVERGED."""
    batch = inputs.scan_batch(4096)
    A0, B0, st0, it0, _, x_off = _solve_scan(batch, 0)
    A1, B1, st1, it1, s1, _ = _solve_scan(batch, 1)
    ok = st0 == 0
    assert np.array_equal(ok, st1 == 0)
    assert np.array_equal(it0[ok], it1[ok])
    pts = np.repeat(ok, np.diff(x_off))
    assert np.array_equal(A0[pts], A1[pts]) and np.array_equal(B0[pts], B1[pts])
    stopped = s1["cycle_period"] > 0
    assert np.all(st1[stopped] == Q.QDSE_ERR_NOT_CONVERGED)
    assert np.all(it1[stopped] <= it0[stopped])
    assert np.all(s1["cycle_found_at"][stopped] == it1[stopped])
    # instances the stop did not end behave as without it
    same = ~stopped
    assert np.array_equal(st0[same], st1[same]) and np.array_equal(it0[same], it1[same])


def test_stall_window_of_4000_leaves_the_converged_set_of_the_scan_unchanged():
    """The no-progress stop the benchmark uses (stall_window = 4000: an instance ends
    NOT_CONVERGED after 4000 successive-approximation sweeps without a new lowest relative
    change) on the 4096-instance scan at the same cap (5000 sweeps), against the run without it:
    the same instances converge, to bitwise the same A and B with the same sweep counts (the rule
    only ends instances, it never changes an iterate), every instance it changed ends
    NOT_CONVERGED before the cap, and fewer instance-sweeps are spent.  On this scan the longest
    stall of a converging instance is 3722 sweeps."""
    batch = inputs.scan_batch(4096)
    A0, B0, st0, it0, s0, x_off = _solve_scan(batch, 1)
    A1, B1, st1, it1, s1, _ = _solve_scan(batch, 1, stall_window=4000)
    ok = st0 == 0
    assert np.array_equal(ok, st1 == 0)
    assert np.array_equal(it0[ok], it1[ok])
    pts = np.repeat(ok, np.diff(x_off))
    assert np.array_equal(A0[pts], A1[pts]) and np.array_equal(B0[pts], B1[pts])
    assert s0["longest_stall"][ok].max() < 4000
    changed = (it1 != it0) | (st1 != st0)
    assert np.all(st1[changed] == Q.QDSE_ERR_NOT_CONVERGED) and np.all(it1[changed] < 5000)
    assert it1.sum() < it0.sum()


def _residual(grids, prm, A, B, precompute, monkeypatch, precision=Q.QDSE_FP64_PRE):
    if precompute == "fp64":
        monkeypatch.setenv("QDSE_PRECOMPUTE", "fp64")
    else:
        monkeypatch.delenv("QDSE_PRECOMPUTE", raising=False)
    ctx = Q.Context(grids, precision=precision)
    FA = torch.empty_like(A)
    FB = torch.empty_like(B)
    ctx.qdse_residual(prm, A, B, FA, FB)
    torch.cuda.synchronize()
    out = FA.cpu().numpy(), FB.cpu().numpy(), ctx.layout()
    ctx.close()
    return out


@pytest.mark.parametrize("mode", [Q.QDSE_COLLOCATED, Q.QDSE_STAGGERED])
def test_fp32_pipe_precompute_gives_the_fp64_precompute_map(mode, monkeypatch):
    """The double-float (FP32-pipe) kernel precompute and the FP64 one feed the same FP64 map
    F(x) (hi + lo kernels) to 2e-13 per instance, on a ragged batch of the scan's shapes and
    interactions (both grid modes)."""
    batch = [b for b in inputs.scan_batch(64)][:24]
    grids = [Q.Grid(b.n_p, b.n_theta, b.s_min, b.s_max, mode) for b in batch]
    prm = [[b.D, b.omega, b.m, 0.0] for b in batch]
    n = sum(b.n_p for b in batch)
    rng = np.random.default_rng(17 + mode)
    A = torch.as_tensor(1 + rng.uniform(0, 1.5, n), device="cuda")
    B = torch.as_tensor(rng.uniform(0.01, 0.8, n), device="cuda")
    FA2, FB2, x_off = _residual(grids, prm, A, B, "f2", monkeypatch)
    FA6, FB6, _ = _residual(grids, prm, A, B, "fp64", monkeypatch)
    for b in range(len(batch)):
        sl = slice(x_off[b], x_off[b + 1])
        ea = np.abs(FA2[sl] - FA6[sl]).max() / np.abs(FA6[sl]).max()
        eb = np.abs(FB2[sl] - FB6[sl]).max() / np.abs(FB6[sl]).max()
        assert ea < 2e-13 and eb < 2e-13, (b, ea, eb)


def test_fused_update_gives_bitwise_the_two_launch_results(monkeypatch):
    """The ring sweep that advances each instance itself (one launch per sweep) and the ring sweep
    followed by a separate update launch compute the same arithmetic in the same order: a ragged
    batch of the scan (both FP32 and FP64 phases, converging, cycling and diverging instances)
    ends bitwise equal, with equal statuses and sweep counts."""
    batch = inputs.scan_batch(192)
    res = []
    for fused in ("1", "0"):
        monkeypatch.setenv("QDSE_FUSED_UPDATE", fused)  # 1: one launch per tick
        res.append(_solve_scan(batch, 1, max_iter=3000))
    (A1, B1, s1, i1, _, _), (A0, B0, s0, i0, _, _) = res
    assert np.array_equal(s1, s0) and np.array_equal(i1, i0)
    assert np.array_equal(A1, A0, equal_nan=True) and np.array_equal(B1, B0, equal_nan=True)
    assert (s1 == 0).sum() > 50


def test_slab_and_ring_sweeps_end_bitwise_equal(monkeypatch):
    """The slab sweep and the per-group ring sweep run the same tile arithmetic in the same order
    for every row group: a ragged batch of the scan solved with each ends bitwise equal, with the
    same statuses and sweep counts (FP32 Picard, tangent and FP64 phases all visited)."""
    batch = inputs.scan_batch(160)
    res = []
    for kind in ("slab", "ring"):
        monkeypatch.setenv("QDSE_SWEEP", kind)
        res.append(_solve_scan(batch, 1, max_iter=2500))
    (A1, B1, s1, i1, _, _), (A0, B0, s0, i0, _, _) = res
    assert np.array_equal(s1, s0) and np.array_equal(i1, i0)
    assert np.array_equal(A1, A0, equal_nan=True) and np.array_equal(B1, B0, equal_nan=True)
    assert (s1 == 0).sum() > 40


@pytest.mark.parametrize("shape", ["8x3", "6x4"])
def test_ring_shapes_end_bitwise_equal(shape, monkeypatch):
    """Ring shapes differ only in which warp takes a row group and how far its copies run ahead;
    each group's tile arithmetic is the same, so a ragged batch of the scan ends bitwise equal to
    the default 12 x 2 shape, with the same statuses and sweep counts."""
    batch = inputs.scan_batch(160)
    res = []
    for s in (shape, "12x2"):
        monkeypatch.setenv("QDSE_RING", s)
        res.append(_solve_scan(batch, 1, max_iter=2500))
    (A1, B1, s1, i1, _, _), (A0, B0, s0, i0, _, _) = res
    assert np.array_equal(s1, s0) and np.array_equal(i1, i0)
    assert np.array_equal(A1, A0, equal_nan=True) and np.array_equal(B1, B0, equal_nan=True)


def test_fp32_only_solve_ends_at_a_fixed_point_or_a_found_cycle():
    """FP32-only Picard to tol = 0 cannot stop on the change unless an iterate repeats exactly:
    every instance of a small batch at the paper's interaction ends before the sweep cap, either
    QDSE_OK at an exact FP32 fixed point (its repeat, period 1, is a fixed point and not a stop) or
    QDSE_ERR_NOT_CONVERGED with the cycle its rounding fell into (period >= 2, found at the sweep
    that ended it).  This runs the cycle stop's detection on real iterates."""
    batch = [inputs.Instance(n, 32, 0.55, 0.678, m) for n in (64, 96, 128)
             for m in (0.0, 0.005, 0.05)]
    grids = [Q.Grid(b.n_p, b.n_theta, b.s_min, b.s_max) for b in batch]
    ctx = Q.Context(grids, precision=Q.QDSE_FP32, tol=0.0, max_iter=20000, stop_cycles=1)
    n = ctx.n_total
    A = torch.ones(n, dtype=torch.float64, device="cuda")
    B = torch.full((n,), 0.3, dtype=torch.float64, device="cuda")
    st = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
    it = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
    ctx.qdse_solve([[b.D, b.omega, b.m, 0.0] for b in batch], A, B, it, st)
    st, it = st.cpu().numpy(), it.cpu().numpy()
    s = ctx.qdse_last_instance_stats()
    ctx.close()
    assert np.all(it < 20000)
    for k in range(len(batch)):
        if st[k] == Q.QDSE_OK:
            assert s["cycle_period"][k] in (0, 1)  # 1: the repeat of the fixed point itself
        else:
            assert st[k] == Q.QDSE_ERR_NOT_CONVERGED
            assert s["cycle_period"][k] >= 2 and s["cycle_found_at"][k] == it[k]


def test_autotune_keeps_a_kernel_with_bitwise_the_same_solves():
    """qdse_autotune solves a ragged batch of the scan once with each of the five FP32 sweep kernels
    (capped at 300 sweeps) and keeps the fastest; the full solve that follows is bitwise the solve
    of a context left at the default kernel (the candidates differ only in how row groups reach
    the SMs), and the start is not modified."""
    batch = inputs.scan_batch(160)
    grids = [Q.Grid(b.n_p, b.n_theta, b.s_min, b.s_max) for b in batch]
    prm = [[b.D, b.omega, b.m, 0.0] for b in batch]
    tuned = Q.Context(grids, precision=Q.QDSE_MIXED, tol=1e-10, max_iter=2500)
    n = tuned.n_total
    A0 = torch.ones(n, dtype=torch.float64, device="cuda")
    B0 = torch.full((n,), 0.3, dtype=torch.float64, device="cuda")
    choice, ms = tuned.qdse_autotune(prm, A0, B0, 300)
    assert 0 <= choice < 5 and ms[choice] > 0 and ms[choice] == min(m for m in ms if m > 0)
    assert torch.all(A0 == 1.0) and torch.all(B0 == 0.3)
    st = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
    it = torch.zeros(len(batch), dtype=torch.int32, device="cuda")
    tuned.qdse_solve(prm, A0, B0, it, st)
    got = (A0.cpu().numpy(), B0.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy())
    tuned.close()
    A, B, s0, i0, _, _ = _solve_scan(batch, 1, max_iter=2500)
    assert np.array_equal(got[2], s0) and np.array_equal(got[3], i0)
    assert np.array_equal(got[0], A, equal_nan=True) and np.array_equal(got[1], B, equal_nan=True)


def test_narrow_group_sweep_gives_bitwise_the_ring_results(monkeypatch):
    """Row groups whose band is at most 32 columns go to their own kernel (four groups per warp,
    eight lanes each) instead of the ring sweep; against the ring alone (QDSE_NARROW=0) the mixed
    solve of 256 scan instances to a cap of 400 sweeps ends bitwise the same: A, B, statuses,
    sweep counts and per-instance records."""
    batch = inputs.scan_batch(256)
    monkeypatch.setenv("QDSE_NARROW", "0")
    ref = _solve_scan(batch, 1, max_iter=400)
    monkeypatch.delenv("QDSE_NARROW", raising=False)
    got = _solve_scan(batch, 1, max_iter=400)
    for a, b in zip(ref[:4], got[:4]):
        assert np.array_equal(a, b)
    for k in ("fp32_sweeps", "fp64_sweeps", "longest_stall", "phase"):
        assert np.array_equal(ref[4][k], got[4][k]), k

