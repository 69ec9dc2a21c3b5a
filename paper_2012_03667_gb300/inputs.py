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


def mscan_batch(n_inst: int = 1024, seed: int = SCAN_SEED, n: int = 512, n_theta: int = 128,
                D: float = 0.55, omega: float = 0.678,
                m_range=(0.0, 0.2)) -> List[Instance]:
    """A current-mass scan that shares one kernel matrix: one grid (N_q = n, N_theta) and the
    paper's Sec. IV interaction for every instance, m ~ U[0, 0.2] GeV from SplitMix64(seed)."""
    rng = SplitMix64(seed ^ 0x6D5343414E)
    return [Instance(n, n_theta, D, omega, m_range[0] + (m_range[1] - m_range[0]) * rng.uniform())
            for _ in range(n_inst)]


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


@dataclass
class MuWorkload:
    """A finite chemical potential sweep workload: external points (p_abs, p4) [n_ext], the nodes
    of the internal product grid (q_abs [n_r] x q4 [n_4]; |q| and |q_4| are Gauss-Legendre nodes
    log-mapped onto [lo, hi]), the cosine nodes z (Gauss-Legendre on [-1, 1]), the chemical
    potentials mu [n_mu] and the interaction.  Nodes only: each side forms its own weights."""
    p_abs: np.ndarray
    p4: np.ndarray
    q_abs: np.ndarray
    q4: np.ndarray
    z: np.ndarray
    mu: np.ndarray
    D: float
    omega: float
    m: float
    lo: float
    hi: float
    T: float = 0.0  # > 0: q4 and p4 are fermion Matsubara frequencies of this temperature


def _log_gl_nodes(n: int, lo: float, hi: float) -> np.ndarray:
    """n Gauss-Legendre nodes log-mapped onto [lo, hi]."""
    t, _ = np.polynomial.legendre.leggauss(n)
    a, b = np.log(lo), np.log(hi)
    return np.exp(a + 0.5 * (t + 1.0) * (b - a))


def mu_workload(n_r: int = 128, n_4: int = 128, n_z: int = 64, n_mu: int = 256,
                seed: int = SCAN_SEED, lo: float = 1e-2, hi: float = 1e2,
                mu_range: Tuple[float, float] = (0.0, 0.4), D: float = 0.93, omega: float = 0.5,
                m: float = 0.005) -> MuWorkload:
    """The finite-mu workload: |q| on n_r Gauss-Legendre nodes log-mapped onto [lo, hi] GeV, q_4 on
    n_4 such nodes and their mirror images (2 n_4 values, symmetric about 0), n_z Gauss-Legendre
    cosine nodes.  External points are staggered between the internal ones: |p|_1 = lo and
    ln |p|_i = (ln q_{i-1} + ln q_i)/2, likewise p_4 > 0 from the positive q_4 nodes, so
    n_ext = n_r * n_4 and no external point is an internal one.  mu ~ U[mu_range] from
    SplitMix64(seed ^ 0x6D75), in draw order."""
    qr = _log_gl_nodes(n_r, lo, hi)
    q4p = _log_gl_nodes(n_4, lo, hi)
    q4 = np.concatenate([-q4p[::-1], q4p])
    stag = lambda x: np.concatenate([[lo], np.sqrt(x[:-1] * x[1:])])
    PR, P4 = np.meshgrid(stag(qr), stag(q4p), indexing="ij")
    z, _ = np.polynomial.legendre.leggauss(n_z)
    rng = SplitMix64(seed ^ 0x6D75)
    mu = np.array([mu_range[0] + (mu_range[1] - mu_range[0]) * rng.uniform() for _ in range(n_mu)])
    return MuWorkload(PR.ravel(), P4.ravel(), qr, q4, z, mu, D, omega, m, lo, hi)


def matsubara_workload(T: float, n_r: int = 128, n_4: int = 32, n_z: int = 64, n_mu: int = 16,
                       seed: int = SCAN_SEED, lo: float = 1e-2, hi: float = 1e2,
                       mu_range: Tuple[float, float] = (0.0, 0.3), D: float = 0.55,
                       omega: float = 0.678, m: float = 0.005) -> MuWorkload:
    """A finite-temperature workload: |q| on n_r Gauss-Legendre nodes log-mapped onto [lo, hi] GeV,
    q_4 on the 2 n_4 fermion Matsubara frequencies +-(2n + 1) pi T (n < n_4), n_z Gauss-Legendre
    cosine nodes.  External points: |p| staggered between the internal |q| as in mu_workload
    (|p|_1 = lo, ln |p|_i = (ln q_{i-1} + ln q_i)/2) times the n_4 positive frequencies, so an
    external point never coincides with an internal one.  mu ~ U[mu_range] from
    SplitMix64(seed ^ 0x54), in draw order.  Nodes only: each side forms its own weights."""
    qr = _log_gl_nodes(n_r, lo, hi)
    wn = (2.0 * np.arange(n_4) + 1.0) * np.pi * T
    q4 = np.concatenate([-wn[::-1], wn])
    PR, P4 = np.meshgrid(np.concatenate([[lo], np.sqrt(qr[:-1] * qr[1:])]), wn, indexing="ij")
    z, _ = np.polynomial.legendre.leggauss(n_z)
    rng = SplitMix64(seed ^ 0x54)
    mu = np.array([mu_range[0] + (mu_range[1] - mu_range[0]) * rng.uniform() for _ in range(n_mu)])
    return MuWorkload(PR.ravel(), P4.ravel(), qr, q4, z, mu, D, omega, m, lo, hi, T)


def mu_iterate(v_abs: np.ndarray, v4: np.ndarray, mu: float, m: float = 0.005) -> np.ndarray:
    """A smooth synthetic iterate (A, C, B) [3, n] at points (|v|, v_4) for chemical potential mu:
    rational functions of s = |v|^2 + (v_4 + i mu)^2 shaped like a dressed propagator,
    A = 1 + 0.6/(1 + s/0.5), C = A (1 + 0.1/(1 + |v|)), B = 0.5/(1 + s/0.8) + m."""
    s = v_abs ** 2 + (v4 + 1j * mu) ** 2
    A = 1.0 + 0.6 / (1.0 + s / 0.5)
    return np.array([A, A * (1.0 + 0.1 / (1.0 + v_abs)), 0.5 / (1.0 + s / 0.8) + m])
