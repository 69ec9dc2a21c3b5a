"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Holds only random draws and workload shapes; none of the solver's arithmetic.  Random numbers come
from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", 2014):
state += 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds; uniform doubles take the top 53
bits.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

MASK = (1 << 64) - 1
SCAN_SEED = 20120366


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


@dataclass
class Instance:
    n_p: int
    n_theta: int
    D: float
    omega: float
    m: float
    s_min: float = 1e-4
    s_max: float = 1e4


# vacuum gap equation, 64 log-mapped GL points on [1e-4, 1e4] GeV^2, 32 angle nodes,
# D = 0.93 GeV^2, w = 0.5 GeV, m = 5 MeV; start A = 1, B = 0.3 GeV; tolerance 1e-10
SMALL = Instance(64, 32, 0.93, 0.5, 0.005)
# same equation at N_p = N_q = 512, N_theta = 128
LARGE = Instance(512, 128, 0.93, 0.5, 0.005)
# the paper's numerical section (Sec. IV): D = 0.55, w = 0.678
PAPER = Instance(64, 32, 0.55, 0.678, 0.005)
A0, B0 = 1.0, 0.3


def scan_batch(n_inst: int = 4096, seed: int = SCAN_SEED,
               n_choices: Tuple[int, ...] = (128, 256, 384, 512),
               theta_choices: Tuple[int, ...] = (32, 64, 128),
               m_range=(0.0, 0.2), omega_range=(0.4, 0.6), D_range=(0.6, 1.2)) -> List[Instance]:
    """The batched mass/interaction scan: per instance m ~ U[0, 0.2] GeV, w ~ U[0.4, 0.6] GeV,
    D ~ U[0.6, 1.2] GeV^2, N_q uniform in {128, 256, 384, 512}, N_theta uniform in
    {32, 64, 128}, drawn in that order from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_inst):
        m = m_range[0] + (m_range[1] - m_range[0]) * rng.uniform()
        w = omega_range[0] + (omega_range[1] - omega_range[0]) * rng.uniform()
        D = D_range[0] + (D_range[1] - D_range[0]) * rng.uniform()
        n = n_choices[min(int(rng.uniform() * len(n_choices)), len(n_choices) - 1)]
        t = theta_choices[min(int(rng.uniform() * len(theta_choices)), len(theta_choices) - 1)]
        out.append(Instance(n, t, D, w, m))
    return out


def adjoint_batch(n_inst: int = 1024, seed: int = SCAN_SEED) -> List[Instance]:
    """The adjoint workload: the scan generator restricted to N_q = 256, N_theta = 64."""
    return scan_batch(n_inst, seed, n_choices=(256,), theta_choices=(64,))


def subsample(batch: List[Instance], k: int, seed: int = SCAN_SEED) -> List[int]:
    """Deterministic subsample of k instance indices covering every (N_q, N_theta) pair first."""
    rng = SplitMix64(seed ^ 0x5DEECE66D)
    by_shape = {}
    for i, inst in enumerate(batch):
        by_shape.setdefault((inst.n_p, inst.n_theta), []).append(i)
    picks = [v[0] for _, v in sorted(by_shape.items())][:k]
    rest = [i for i in range(len(batch)) if i not in set(picks)]
    while len(picks) < min(k, len(batch)):
        j = int(rng.uniform() * len(rest))
        picks.append(rest.pop(j))
    return sorted(picks)


def params_array(batch: List[Instance]) -> np.ndarray:
    """(n, 4) array of (D, omega, m, mu = 0)."""
    return np.array([[b.D, b.omega, b.m, 0.0] for b in batch], dtype=np.float64)
