"""Benchmark: batched solves of the BC-vertex quark gap equation on GB300.

Workload (default ``scan``): the batched mass/interaction scan of 4096 instances (m ~ U[0, 0.2] GeV,
w ~ U[0.4, 0.6] GeV, D ~ U[0.6, 1.2] GeV^2, N_q in {128, 256, 384, 512}, N_theta in {32, 64, 128},
SplitMix64 seed 20120366), log-mapped GL grids on [1e-4, 1e4] GeV^2, start A = 1, B = 0.3 GeV,
tolerance 1e-10 (relative change, Eq. jifenab2).  One step = one complete batched solve: angular
kernel precompute, FP32 sweeps, FP64 residuals and refinement, for every instance.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the host cores
on a bounded subsample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BC-kernel evals/s per sweep; batched solves/s at 1e-8 rel err vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scan",
                    choices=["scan", "large", "small", "adjoint", "mu", "mu-small", "mu-solve",
                             "table1"],
                    help="scan: 4096-instance mass/interaction scan (default); large/small: one "
                         "N = 512 / N = 64 instance; adjoint: 1024 scan instances at N_q = 256, "
                         "N_theta = 64, forward solve + condensate gradient by the adjoint; mu: "
                         "finite-mu batched sweep, 256 mu on the full grid; mu-small: a small "
                         "case of it; mu-solve: finite-mu solve of 32 mu; table1: Sec. IV "
                         "Table 1 (with --impl reference, the four CPU algorithms)")
    ap.add_argument("--n-inst", type=int, default=4096)
    ap.add_argument("--max-iter", type=int, default=5000)
    ap.add_argument("--check", type=int, default=8,
                    help="instances re-solved by the plain FP64 GPU form for the accuracy check")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mu-d", type=float, default=0.55, help="D of --workload mu-solve")
    ap.add_argument("--mu-omega", type=float, default=0.678, help="omega of --workload mu-solve")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
def workload(args, rank=0):
    from paper_2012_03667_gb300 import inputs
    if args.workload == "scan":
        batch = inputs.scan_batch(args.n_inst, seed=inputs.SCAN_SEED + rank)
        name = (f"batched mass/interaction scan, {args.n_inst} instances, N_q in "
                "{128,256,384,512}, N_theta in {32,64,128}, BC vertex")
    elif args.workload == "large":
        batch = [inputs.LARGE]
        name = "single instance N_p = N_q = 512, N_theta = 128, D = 0.93, w = 0.5, m = 5 MeV"
    else:
        batch = [inputs.SMALL]
        name = "single instance N = 64, N_theta = 32, D = 0.93, w = 0.5, m = 5 MeV"
    return batch, name


def band_fraction(batch):
    """Share of the dense N_p x N_q kernel entries inside the bands the precompute keeps: pairs
    with (sqrt P - sqrt Q)^2 / omega^2 < 70 on each instance's collocated log-mapped
    Gauss-Legendre grid (every other pair carries exp(-k^2/omega^2) <= exp(-70) at every
    angle and is stored as an exact zero, never read by the sweeps).  Host arithmetic only."""
    kept = dense = 0.0
    dist = {}
    for b in batch:
        key = (b.n_p, b.s_min, b.s_max)
        if key not in dist:  # sorted |sqrt P - sqrt Q| over all pairs of this grid
            t, _ = np.polynomial.legendre.leggauss(b.n_p)
            u0, u1 = np.log(b.s_min), np.log(b.s_max)
            r = np.sqrt(np.exp(0.5 * (u1 + u0) + 0.5 * (u1 - u0) * t))
            dist[key] = np.sort(np.abs(r[:, None] - r[None, :]).ravel())
        kept += float(np.searchsorted(dist[key], np.sqrt(70.0) * b.omega, side="left"))
        dense += float(b.n_p) ** 2
    return kept / dense


def evals_per_sweep(batch):
    return float(sum(b.n_p * b.n_p * b.n_theta for b in batch))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.stop = threading.Event()
        self.th = None

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        if self.th:
            self.th.join(timeout=6)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 3 + k and r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


PROFILE = os.path.join(ROOT, "profiles", "k_tick_ring_scan256.md")


def traffic_ratio():
    """DRAM bytes per algorithmic byte of the FP32 sweep kernel, from the ncu capture summarised in
    profiles/ (a 256-instance tick of the same scan; traffic grows in proportion to the kernel
    entries a launch reads, so it scales to any launch by the algorithmic bytes)."""
    try:
        with open(PROFILE) as f:
            for line in f:
                if line.startswith("traffic_per_algorithmic_byte:"):
                    return float(line.split(":", 1)[1])
    except (OSError, ValueError):
        pass
    return None


def job_rate(ms_local, ok_local, steps, world, device):
    """Whole-job figures over all ranks (weak scaling: every rank solves its own batch): the
    slowest rank's time, the converged solves summed over ranks, and their rate.  Returns
    (ms, total_ok, solves_per_s)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    n = torch.tensor([float(ok_local)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    total = float(n.item())
    return ms, total, total * steps / (ms / 1e3)


# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2012_03667_gb300 import qdse as Q

    batch, name = workload(args, rank)
    grids = [Q.Grid(b.n_p, b.n_theta, b.s_min, b.s_max) for b in batch]
    prm = [[b.D, b.omega, b.m, 0.0] for b in batch]
    ctx = Q.Context(grids, precision=Q.QDSE_MIXED, tol=1e-10, max_iter=args.max_iter)
    nt = ctx.n_total
    dev = torch.device("cuda", local)
    A = torch.ones(nt, dtype=torch.float64, device=dev)
    B = torch.full((nt,), 0.3, dtype=torch.float64, device=dev)
    iters = torch.zeros(len(batch), dtype=torch.int32, device=dev)
    status = torch.zeros(len(batch), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        A.fill_(1.0)
        B.fill_(0.3)
        ctx.qdse_solve(prm, A, B, iters, status)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = 0
    prof = {"precompute": [0.0, 0], "sweep": [0.0, 0], "update": [0.0, 0], "other": [0.0, 0]}
    work = {"sweep_bytes": 0.0, "kernel_evals": 0.0}
    sweeps32 = sweeps64 = 0
    ctx.qdse_set_profiling(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
            st_ = ctx.qdse_last_stats()
            launches += st_["kernel_launches"]
            sweeps32 += st_["fp32_sweeps"]
            sweeps64 += st_["fp64_sweeps"]
            for k, v in ctx.qdse_profile().items():
                prof[k][0] += v["ms"]
                prof[k][1] += v["launches"]
            for k, v in ctx.qdse_last_work().items():
                work[k] += v
        ev1.record(stream)
        torch.cuda.synchronize()
    ctx.qdse_set_profiling(False)
    ms = ev0.elapsed_time(ev1)
    st = status.cpu().numpy()
    it = iters.cpu().numpy()
    ok = int((st == 0).sum())
    ms, _, solves_per_s = job_rate(ms, ok, args.steps, world, dev)

    # end to end through the host-buffer entry point (copies in the timed region)
    Ah = np.ones(nt)
    Bh = np.full(nt, 0.3)
    t0 = time.perf_counter()
    ctx.qdse_solve_host(prm, Ah, Bh)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ok * world / e2e_s, "unit": "solves/s",
           "h2d_bytes_per_step": int(2 * nt * 8), "d2h_bytes_per_step": int(2 * nt * 8)}

    # accuracy: sampled instances checked against the plain FP64 (on-the-fly) GPU form.  The
    # plain FP64 successive approximation restarted from the mixed-precision solution must stay
    # within 1e-8 of it (the solution is an FP64 fixed point to that accuracy); where the plain
    # FP64 solve from the common start converges to the same fixed point, that is compared too.
    acc = None
    if rank == 0 and args.check > 0:
        from paper_2012_03667_gb300 import inputs
        idx = inputs.subsample(batch, min(args.check, len(batch))) if len(batch) > 1 else [0]
        x_off = ctx.layout()
        Ah = A.cpu().numpy()
        Bh = B.cpu().numpy()
        worst, checked, same_start, worst_start = 0.0, 0, 0, 0.0

        def err(a, b, ra, rb):
            return max(np.abs(a - ra).max() / np.abs(ra).max(),
                       np.abs(b - rb).max() / np.abs(rb).max(),
                       np.abs(b / a - rb / ra).max() / np.abs(rb / ra).max())

        for i in idx:
            if st[i] != 0:
                continue
            b = batch[i]
            sl = slice(x_off[i], x_off[i + 1])
            c64 = Q.Context(Q.Grid(b.n_p, b.n_theta, b.s_min, b.s_max), 1, precision=Q.QDSE_FP64,
                            tol=1e-10, max_iter=args.max_iter)
            s64 = torch.zeros(1, dtype=torch.int32, device=dev)
            a64 = torch.as_tensor(Ah[sl], device=dev).contiguous()
            b64 = torch.as_tensor(Bh[sl], device=dev).contiguous()
            c64.qdse_solve([prm[i]], a64, b64, None, s64)
            if int(s64.item()) == 0:
                checked += 1
                worst = max(worst, err(Ah[sl], Bh[sl], a64.cpu().numpy(), b64.cpu().numpy()))
            a64.fill_(1.0)
            b64.fill_(0.3)
            c64.qdse_solve([prm[i]], a64, b64, None, s64)
            if int(s64.item()) == 0:
                e = err(Ah[sl], Bh[sl], a64.cpu().numpy(), b64.cpu().numpy())
                if e < 1e-6:
                    same_start += 1
                    worst_start = max(worst_start, e)
            c64.close()
        acc = {"sampled": len(idx), "verified_fp64_fixed_point": checked,
               "max_rel_err_vs_fp64_restart": worst,
               "same_fixed_point_as_fp64_from_start": same_start,
               "max_rel_err_vs_fp64_from_start": worst_start}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, batch)

    if rank == 0:
        hbm, kind = peaks()
        sweep_ms, sweep_n = prof["sweep"]
        achieved = work["sweep_bytes"] / (sweep_ms / 1e3) / 1e9 if sweep_ms > 0 else None
        ratio = traffic_ratio()
        traffic = ratio * work["sweep_bytes"] / max(sweep_n, 1) if ratio else None
        shares = {k: v[0] for k, v in prof.items()}
        tot = sum(shares.values()) or 1.0
        line = {
            "metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": name, "instances_per_gpu": len(batch),
                       "evals_per_sweep": evals_per_sweep(batch), "tol": 1e-10,
                       "max_sweeps": args.max_iter, "precision": "mixed (FP32 sweeps, FP64 "
                       "residual + refinement)",
                       "l2": "inputs larger than L2: the 6 GB kernel pool is re-read each sweep"},
            "converged": ok, "mean_sweeps": float(it.mean()), "max_sweeps": int(it.max()),
            "kernel_evals_per_s": work["kernel_evals"] / (ms / 1e3),
            "kernel_evals_per_s_sweep_only": (work["kernel_evals"] / (sweep_ms / 1e3)
                                              if sweep_ms > 0 else None),
            "sweeps": {"fp32_instance_sweeps": sweeps32, "fp64_instance_sweeps": sweeps64},
            "e2e": e2e, "gpu_launches": launches, "accuracy": acc,
            "roofline": {"kernel": "k_tick_ring (batched FP32 sweep)", "bound": "hbm",
                         "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                         "traffic_unit": "bytes per launch (ncu ratio x algorithmic bytes)",
                         "peak_kind": kind, "launches": sweep_n,
                         "avg_launch_ms": sweep_ms / max(sweep_n, 1),
                         "alg_bytes_per_launch": work["sweep_bytes"] / max(sweep_n, 1)},
            "device_time_share": {k: v / tot for k, v in shares.items()},
            "clocks": clk.summary(),
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        try:  # reporting only: never let it cost the line
            line["band"] = {"kept_fraction_of_dense": band_fraction(batch),
                            "criterion": "(sqrt P - sqrt Q)^2 / omega^2 < 70; the rest are "
                                         "exact zeros the sweeps never read"}
        except Exception as e:  # pragma: no cover
            line["band"] = {"error": str(e)}
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
def oracle_sample(args, batch, seconds):
    """Solve a bounded sample of the workload with the FP64 CPU oracle on every host core."""
    from oracle import oracle as O
    from paper_2012_03667_gb300 import inputs
    O.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    idx = inputs.subsample(batch, min(64, len(batch))) if len(batch) > 1 else [0]
    idx = sorted(idx, key=lambda i: batch[i].n_p * batch[i].n_p * batch[i].n_theta)
    t0 = time.perf_counter()
    solved, used = 0, []
    for i in idx:
        b = batch[i]
        pr = O.Problem(n=b.n_p, n_theta=b.n_theta, s_min=b.s_min, s_max=b.s_max, D=b.D,
                       omega=b.omega, m=b.m)
        _, _, _, _, st = O.solve(pr, tol=1e-10, max_iter=args.max_iter, nthreads=cores)
        solved += int(st == 0)
        used.append(i)
        if time.perf_counter() - t0 > seconds:
            break
    return solved, time.perf_counter() - t0, used, cores


def cpu_baseline(args, batch):
    solved, t, used, cores = oracle_sample(args, batch, args.cpu_seconds)
    return {"value": solved / t, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(used)} instances of the deterministic 64-instance subsample "
                      f"(smallest grids first), FP64 successive approximation to 1e-10, "
                      f"OpenMP over the external index, {t:.1f} s"}


def run_reference(args):
    """The FP64 CPU oracle (plain triple loop, OpenMP over the external index) on host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    batch, name = workload(args)
    if args.warmup > 0:
        oracle_sample(args, batch, min(args.cpu_seconds, 5.0))
    tot_s, tot_t, used, cores = 0, 0.0, [], 1
    for _ in range(args.steps):
        s_, t_, used, cores = oracle_sample(args, batch, args.cpu_seconds)
        tot_s += s_
        tot_t += t_
    v = tot_s / tot_t
    sample = (f"{len(used)} instances of the deterministic 64-instance subsample (smallest grids "
              f"first) per step, FP64 successive approximation to 1e-10")
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": name, "max_sweeps": args.max_iter},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------------
# Table 1 of Sec. IV: N = 150 radial points, M = 100 angular nodes, xi = 0.005, the paper's
# interaction D = 0.55, omega = 0.678 (Intel Core i7 at 1.00 GHz, GCC 9.3.0, 11 iterations).
TABLE1 = dict(n=150, n_theta=100, tol=0.005, D=0.55, omega=0.678, m=0.005)
TABLE1_PAPER = {"1 traditional, serial": {"cpu_s": 65, "cpu_pct": 100.0},
                "2 modified, serial": {"cpu_s": 6, "cpu_pct": 100.0},
                "3 traditional, parallel": {"cpu_s": 9, "cpu_pct": 782.0},
                "4 modified, parallel": {"cpu_s": 1, "cpu_pct": 792.0}}


def run_table1(args):
    """Table 1 of Sec. IV on this machine.  --impl reference: the paper's four CPU algorithms
    (traditional or modified interpolation, serial or OpenMP over the external index on every
    host core) by the FP64 oracle on the staggered grid, to the relative change xi = 0.005 (R7);
    the value is algorithm 4's time.  --impl ours: the GPU solver on the same problem, plain FP64
    sweeps to the same xi and mixed precision to 1e-10 (times from CUDA events)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t = TABLE1
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    if args.impl == "reference":
        from oracle import oracle as O
        O.build()
        algs = {}
        for name, mode, nt in (("1 traditional, serial", O.STAGGERED_TRADITIONAL, 1),
                               ("2 modified, serial", O.STAGGERED, 1),
                               ("3 traditional, parallel", O.STAGGERED_TRADITIONAL, cores),
                               ("4 modified, parallel", O.STAGGERED, cores)):
            pr = O.Problem(n=t["n"], n_theta=t["n_theta"], grid_mode=mode, D=t["D"],
                           omega=t["omega"], m=t["m"])
            w0, c0 = time.perf_counter(), time.process_time()
            A, B, it, ch, st = O.solve(pr, tol=t["tol"], max_iter=1000, nthreads=nt)
            wall, cpu = time.perf_counter() - w0, time.process_time() - c0
            algs[name] = {"wall_s": wall, "cpu_pct": 100.0 * cpu / wall, "threads": nt,
                          "iterations": it, "status": st, "A0": A[0], "M0": B[0] / A[0]}
        v = algs["4 modified, parallel"]["wall_s"]
        line = {"metric": "Table 1 solve time (Sec. IV)", "value": v, "unit": "s",
                "n_gpus": 0, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * v,
                "higher_is_better": False, "scaling": "none", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": "Table 1: N = 150, M = 100 (Gauss-Chebyshev), xi = 0.005 "
                                       "relative change, D = 0.55, omega = 0.678, m = 0.005, "
                                       "staggered grid on [1e-4, 1e4] GeV^2"},
                "algorithms": algs, "cores": cores, "paper": TABLE1_PAPER,
                "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                                 "sample": "the whole Table 1 problem, algorithm 4"},
                "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_03667_gb300 import qdse as Q
    grid = Q.Grid(t["n"], t["n_theta"], 1e-4, 1e4, Q.QDSE_STAGGERED)
    prm = [[t["D"], t["omega"], t["m"], 0.0]]
    out = {}
    for name, prec, tol in (("fp64 sweeps to xi", Q.QDSE_FP64, t["tol"]),
                            ("mixed to 1e-10", Q.QDSE_MIXED, 1e-10)):
        ctx = Q.Context(grid, 1, precision=prec, tol=tol)
        A = torch.ones(t["n"], dtype=torch.float64, device="cuda")
        B = torch.full((t["n"],), 0.3, dtype=torch.float64, device="cuda")
        it = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        times = []
        for rep in range(args.warmup + args.steps):
            A.fill_(1.0)
            B.fill_(0.3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            ctx.qdse_solve(prm, A, B, it, st)
            e1.record()
            torch.cuda.synchronize()
            if rep >= args.warmup:
                times.append(e0.elapsed_time(e1) / 1e3)
        out[name] = {"s": float(np.median(times)), "iterations": int(it.item()),
                     "status": int(st.item()), "A0": float(A[0].item()),
                     "M0": float((B[0] / A[0]).item())}
        ctx.close()
    v = out["fp64 sweeps to xi"]["s"]
    line = {"metric": "Table 1 solve time (Sec. IV)", "value": v, "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * v,
            "higher_is_better": False, "scaling": "none", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "Table 1: N = 150, M = 100 (Gauss-Chebyshev), xi = 0.005 "
                                   "relative change, D = 0.55, omega = 0.678, m = 0.005, "
                                   "staggered grid on [1e-4, 1e4] GeV^2"},
            "gpu": out, "paper": TABLE1_PAPER}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------------
def run_adjoint(args):
    """Gradients of the chiral condensate -<qq> of every instance with respect to (m, D, w, mu):
    one step = forward mixed-precision solve to 1e-12 (kernel precompute included) + condensate
    cotangent + adjoint solve (dK/dw precompute included).  Single GPU; other ranks idle."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_03667_gb300 import inputs
    from paper_2012_03667_gb300 import qdse as Q
    n = args.n_inst if args.n_inst != 4096 else 1024
    batch = inputs.adjoint_batch(n, seed=inputs.SCAN_SEED + rank)
    grids = [Q.Grid(b.n_p, b.n_theta, b.s_min, b.s_max) for b in batch]
    prm = [[b.D, b.omega, b.m, 0.0] for b in batch]
    ctx = Q.Context(grids, precision=Q.QDSE_MIXED, tol=1e-12, max_iter=args.max_iter)
    nt = ctx.n_total
    dev = torch.device("cuda", local)
    A = torch.ones(nt, dtype=torch.float64, device=dev)
    B = torch.full((nt,), 0.3, dtype=torch.float64, device=dev)
    st = torch.zeros(n, dtype=torch.int32, device=dev)
    ist = torch.zeros(n, dtype=torch.int32, device=dev)
    cbar = torch.ones(n, dtype=torch.float64, device=dev)
    gA, gB = torch.zeros_like(A), torch.zeros_like(B)
    gp = torch.zeros(4 * n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        A.fill_(1.0)
        B.fill_(0.3)
        ctx.set_options(tol=1e-12, max_iter=args.max_iter)
        ctx.qdse_solve(prm, A, B, None, st)
        ctx.qdse_condensate_vjp(A, B, cbar, gA, gB)
        ctx.set_options(tol=1e-12, max_iter=20000)
        ctx.qdse_adjoint(prm, A, B, gA, gB, gp, None, ist)

    for _ in range(args.warmup):
        step()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ok = int(((st.cpu().numpy() == 0) & (ist.cpu().numpy() == 0)).sum())
    if rank != 0:
        return
    line = {"metric": "condensate gradients d(-<qq>)/d(m, D, w, mu) per second "
                      "(forward solve + adjoint, 1e-12)",
            "value": ok * args.steps / (ms / 1e3), "unit": "gradients/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"adjoint: {n} scan instances, N_q = 256, N_theta = 64, "
                                   "BC vertex, mu = 0",
                       "l2": "inputs larger than L2: the kernel pools are re-read each sweep"},
            "gradients_ok": ok, "clocks": clk.summary()}
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------------
# Finite chemical potential: FP32 operations of one (pair, mu) evaluation of the Ball-Chiu sweep
# (csrc/mu_pair.cuh: 118 additions + 159 multiplications + 1 reciprocal in mu_pair_add) and of one
# pair's real combinations, shared by a tile of 8 chemical potentials (12 + 24 + 1 in
# mu_pair_real), counted by instantiating the templates with an operation-counting scalar.
MU_FLOPS_PAIR_MU = 278
MU_FLOPS_PAIR = 37
MU_TILE = 8
# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def mu_cpu_baseline(w, seconds=15.0):
    """The finite-mu FP64 oracle (explicit 4x4 Dirac matrices, OpenMP over external points) on a
    bounded sample of the workload: all internal points and angles for a growing set of external
    points at two chemical potentials, until about `seconds` of CPU work; (pair, mu) evaluations
    per second, pairs counted as all internal points (the oracle keeps no windows)."""
    from oracle import oracle_mu as OM
    from paper_2012_03667_gb300 import inputs
    OM.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    QR, Q4 = np.meshgrid(w.q_abs, w.q4, indexing="ij")
    qv, q4 = QR.ravel(), Q4.ravel()
    evals, t_total, n_pts = 0, 0.0, 0
    n = max(1, cores)
    stride = max(1, len(w.p_abs) // 97)
    for b in (0, len(w.mu) - 1):
        mu = float(w.mu[b])
        Fq = inputs.mu_iterate(qv, q4, mu, w.m)
        idx = np.arange(0, len(w.p_abs), stride)[:n]
        Fp = inputs.mu_iterate(w.p_abs[idx], w.p4[idx], mu, w.m)
        t0 = time.perf_counter()
        OM.sweep(w.p_abs[idx], w.p4[idx], qv, q4, w.w_q, w.z, w.w_z, w.D, w.omega, w.m, mu,
                 *Fp, *Fq, nthreads=cores)
        t_total += time.perf_counter() - t0
        evals += len(idx) * len(qv)
        n_pts += len(idx)
        if t_total > seconds:
            break
    return {"value": evals / t_total, "unit": "pair-mu evals/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{n_pts} external points x all {len(qv)} internal points x "
                      f"{len(w.z)} angles at 2 chemical potentials, FP64, {t_total:.1f} s"}


def run_mu(args):
    """One step = one batched FP32 sweep of the finite-mu gap equation (Ball-Chiu vertex) for all
    chemical potentials: propagator prep + sweep over the precomputed angular-moment table.  The
    table precompute (once per omega and grid) is timed separately.  Single GPU; other ranks
    idle."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_03667_gb300 import inputs
    from paper_2012_03667_gb300 import qdse_mu as QM
    if args.workload == "mu":
        w = inputs.mu_workload()
        name = ("finite mu: 256 mu ~ U[0, 0.4] GeV, |p| 128 x p4 128 external (staggered), "
                "|q| 128 x q4 256 internal, log-mapped GL on [1e-2, 1e2] GeV, 64 GL angles, "
                "D = 0.93, omega = 0.5, m = 0.005, BC vertex, FP32 sweep")
    else:
        w = inputs.mu_workload(n_r=64, n_4=48, n_z=64, n_mu=32)
        name = "finite mu (small): 32 mu, |p| 64 x p4 48, |q| 64 x q4 96, 64 angles, FP32 sweep"
    QR, Q4 = np.meshgrid(w.q_abs, w.q4, indexing="ij")
    qv, q4 = QR.ravel(), Q4.ravel()
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    g = QM.MuGrid(w.p_abs, w.p4, w.q_abs, w.q4, w.w_q, w.z, w.w_z, w.omega, 3)
    t_pre = time.perf_counter() - t0
    info = g.info()
    n_mu = len(w.mu)
    Fe_h = np.stack([inputs.mu_iterate(w.p_abs, w.p4, mu, w.m) for mu in w.mu])
    Fi_h = np.stack([inputs.mu_iterate(qv, q4, mu, w.m) for mu in w.mu])
    Fe = torch.from_numpy(Fe_h).to(dev)
    Fi = torch.from_numpy(Fi_h).to(dev)
    out = torch.empty_like(Fe)
    mu = list(w.mu)
    stream = torch.cuda.current_stream()

    def step():
        g.sweep(mu, w.D, w.m, Fe, Fi, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.profile()
    g.set_profiling(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof = g.profile()
    g.set_profiling(False)
    ok = bool(torch.isfinite(torch.view_as_real(out)).all().item())
    # end to end through the same call: pinned host inputs in, the result out, every step
    Fe_p = torch.from_numpy(Fe_h).pin_memory()
    Fi_p = torch.from_numpy(Fi_h).pin_memory()
    out_p = torch.empty(out.shape, dtype=out.dtype).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        Fe.copy_(Fe_p, non_blocking=True)
        Fi.copy_(Fi_p, non_blocking=True)
        step()
        out_p.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    if rank != 0:
        return
    evals = info["n_pairs"] * n_mu
    sweep_ms = prof["sweep"]["ms"] / max(prof["sweep"]["launches"], 1)
    flops = evals * MU_FLOPS_PAIR_MU + info["n_pairs"] * -(-n_mu // MU_TILE) * MU_FLOPS_PAIR
    achieved = flops / (sweep_ms / 1e3) / 1e12
    line = {"metric": "finite-mu sweep: (pair, mu) evaluations per second",
            "value": evals * args.steps / (ms / 1e3), "unit": "pair-mu evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": name, "n_mu": n_mu, "n_ext": len(w.p_abs),
                       "n_int": len(qv), "pairs_kept": info["n_pairs"],
                       "table_bytes": info["table_bytes"],
                       "l2": "inputs larger than L2: the moment table is re-read each step"},
            "precompute_s": t_pre,
            "kernel_ms": {"prep": prof["prep"]["ms"] / max(prof["prep"]["launches"], 1),
                          "sweep": sweep_ms},
            "roofline": {"bound": "alu", "kernel": "k_mu_sweep<float, 8>",
                         "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None,
                         "flops_per_launch": flops,
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"},
            "e2e": {"value": evals * args.steps / (ms_e2e / 1e3), "unit": "pair-mu evals/s",
                    "h2d_bytes_per_step": Fe_h.nbytes + Fi_h.nbytes,
                    "d2h_bytes_per_step": out_p.numel() * out_p.element_size()},
            "gpu_launches": 2 * args.steps, "outputs_finite": ok, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = mu_cpu_baseline(w, args.cpu_seconds)
    print(json.dumps(line))


def run_mu_reference(args):
    """--impl reference --workload mu: the finite-mu oracle timed on the host cores (rank 0)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from paper_2012_03667_gb300 import inputs
    w = inputs.mu_workload()
    cb = mu_cpu_baseline(w, args.cpu_seconds)
    v = cb["value"]
    line = {"metric": "finite-mu sweep: (pair, mu) evaluations per second", "value": v,
            "unit": "pair-mu evals/s", "n_gpus": args.gpus, "steps": 1, "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "finite mu: the full grid of --workload mu, sampled"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "pair-mu evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_mu_solve(args):
    """One step = solving the finite-mu equation (Ball-Chiu vertex) for 32 chemical potentials on
    the full grid from A = C = 1, B = 0.3: FP32 sweeps to a change of 1e-5, then FP64 sweeps on an
    FP64 table of the same points to 1e-10, at most 200 sweeps.  Interaction: the paper's Sec. IV
    values D = 0.55, omega = 0.678 (with the Ball-Chiu vertex at omega = 0.5 the Nambu solution
    ends at a fold near D = 0.75, so at D = 0.93 the iteration has no physical fixed point to
    reach; --mu-d 0.93 --mu-omega 0.5 runs that case).  Both moment tables are built once, outside
    the timed region.  Single GPU; other ranks idle."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_03667_gb300 import inputs
    from paper_2012_03667_gb300 import qdse_mu as QM
    n_mu = 32
    w = inputs.mu_workload(n_mu=n_mu, D=args.mu_d, omega=args.mu_omega)
    pa, p4a = np.unique(w.p_abs), np.unique(w.p4)
    g32 = QM.MuGrid(pa, p4a, w.q_abs, w.q4, w.w_q, w.z, w.w_z, w.omega, 3, product=True)
    g64 = QM.MuGrid(pa, p4a, w.q_abs, w.q4, w.w_q, w.z, w.w_z, w.omega, 0, product=True)
    dev = torch.device("cuda", local)
    start = np.zeros((n_mu, 3, g32.n_ext), dtype=np.complex128)
    start[:, 0] = start[:, 1] = 1.0
    start[:, 2] = 0.3
    F = torch.from_numpy(start).to(dev)
    mu = list(w.mu)
    stream = torch.cuda.current_stream()
    res = {}

    def step():
        F.copy_(torch.from_numpy(start).to(dev))
        res["iters"], res["status"] = g32.solve(mu, w.D, w.m, F, tol=1e-10, max_iter=200,
                                                vertex=0, refine=g64, switch_tol=1e-5)

    for _ in range(args.warmup):
        step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ok = int((res["status"] == 0).sum())
    if rank != 0:
        return
    line = {"metric": "finite-mu solves per second (BC vertex, 1e-10, FP32 sweeps + FP64 "
                      "refinement)",
            "value": ok * args.steps / (ms / 1e3), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "finite mu solve: 32 mu ~ U[0, 0.4] GeV, |p| 128 x p4 128 "
                                   "external, |q| 128 x q4 256 internal, 64 angles, "
                                   f"D = {w.D}, omega = {w.omega}, m = 0.005, start A = C = 1, "
                                   "B = 0.3",
                       "max_sweeps": 200},
            "converged": ok, "sweeps": [int(x) for x in res["iters"]],
            "status": [int(x) for x in res["status"]], "clocks": clk.summary()}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.workload == "table1":
        run_table1(a)
    elif a.impl == "reference" and a.workload == "mu":
        run_mu_reference(a)
    elif a.impl == "reference":
        run_reference(a)
    elif a.workload == "adjoint":
        run_adjoint(a)
    elif a.workload == "mu-solve":
        run_mu_solve(a)
    elif a.workload.startswith("mu"):
        run_mu(a)
    else:
        run_ours(a)
