"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds no arithmetic of the heat-bath method: it only draws
random numbers with numpy and names the workload shapes.  Both the CUDA path
and the CPU oracle consume what it returns.
"""
from __future__ import annotations

import numpy as np


def random_links(Ns: int, Nt: int, seed: int) -> np.ndarray:
    """Uniformly random unit quaternions, canonical host layout
    float64[V][4][4] = [lex][mu][a0..a3]."""
    rng = np.random.default_rng(seed)
    n = rng.standard_normal((Ns ** 3 * Nt, 4, 4))
    n /= np.linalg.norm(n, axis=2, keepdims=True)
    return np.ascontiguousarray(n)


def random_unit_quaternions(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


# Workload shapes (the paper's benchmark: random SU(2) start, heat-bath
# sweeps with the mean plaquette after each sweep, Sec. 2.1; finite-T scan,
# Sec. 2.2).
SMALL_FP64 = dict(name="8^4 FP64 hot start beta=2.3", Ns=8, Nt=8, beta=2.3, sweeps=100,
                  init_seed=1, hb_seed=1)
MEDIUM = dict(name="32^4 hot start beta=6.0", Ns=32, Nt=32, beta=6.0, sweeps=100,
              init_seed=2, hb_seed=2)
LARGE = dict(name="64^4 hot start beta=2.5", Ns=64, Nt=64, beta=2.5, sweeps=100,
             init_seed=3, hb_seed=3)
HUGE = dict(name="128^4 hot start beta=2.5", Ns=128, Nt=128, beta=2.5, sweeps=100,
            init_seed=3, hb_seed=3)


def temperature_scan(n_points: int = 21, Ns: int = 48, Nt: int = 4):
    """Finite-temperature scan: Ns^3 x Nt lattices, beta = 2.20 .. 2.40 in
    steps of 0.01, per-lattice seeds 1000 + i."""
    return [dict(Ns=Ns, Nt=Nt, beta=round(2.20 + 0.01 * i, 2), seed=1000 + i)
            for i in range(n_points)]


def batched_ensemble(n: int = 64, seed: int = 5):
    """Independent lattices of uneven shape: Ns uniform in {16,24,32,40,48},
    Nt uniform in {4,6,8}, beta uniform in [2.2, 2.6], seeds 5000 + l."""
    rng = np.random.default_rng(seed)
    Ns = rng.choice([16, 24, 32, 40, 48], size=n)
    Nt = rng.choice([4, 6, 8], size=n)
    beta = rng.uniform(2.2, 2.6, size=n)
    return [dict(Ns=int(Ns[i]), Nt=int(Nt[i]), beta=float(beta[i]), seed=5000 + i)
            for i in range(n)]
