"""The N > 1 path of bench.py on CPU: two gloo ranks, no GPU.

Every rank solves its own batch (weak scaling, no data-path collective).  Checked here: the ranks'
batches are distinct and each is deterministic, and the whole-job figures are the slowest rank's
time and the converged solves summed over the ranks.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)

    class A:
        workload, n_inst = "scan", 64
    batch, _ = bench.workload(A, rank)
    again, _ = bench.workload(A, rank)
    ms, total, rate = bench.job_rate(100.0 + 50.0 * rank, 10 + rank, 3, world,
                                     torch.device("cpu"))
    out[rank] = (tuple((b.n_p, b.n_theta, b.D, b.omega, b.m) for b in batch),
                 batch == again, ms, total, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn")
    b0, same0, ms0, tot0, rate0 = out[0]
    b1, same1, ms1, tot1, rate1 = out[1]
    assert same0 and same1                      # each rank's batch is deterministic
    assert b0 != b1 and len(b0) == len(b1) == 64  # ranks draw different instances
    assert ms0 == ms1 == 150.0                  # the slowest rank's time
    assert tot0 == tot1 == 21.0                 # converged solves summed over ranks
    assert rate0 == pytest.approx(21.0 * 3 / 0.150)
