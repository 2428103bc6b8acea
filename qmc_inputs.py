"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle-side checks.

This module holds no arithmetic of the Monte Carlo method (no pair function, potential,
move, estimator or random-number mapping of the method).  It only makes problem inputs:
box sides for a given density, particle positions scattered in the box, and walker
parameter sets with the shapes of the paper's workloads (liquid 4He at 21.86 nm^-3,
b = 3.07 A, N from 2 to 10 000).  Both the CUDA path and the oracle receive the same arrays.
"""
from __future__ import annotations

import numpy as np

RHO_HE = 0.02186          # A^-3: experimental equilibrium density of liquid 4He (paper, Sec. 7)
B_HE = 3.07               # A: optimal Jastrow b of the paper's benchmarks (Sec. 7)
HBAR2_OVER_M = 12.1194    # K A^2 for 4He


def box_side(n: int, rho: float) -> float:
    """Side of the cubic box holding n particles at number density rho."""
    return float((n / rho) ** (1.0 / 3.0))


def jittered_lattice(n: int, L: float, seed: int, sigma: float = 0.25) -> np.ndarray:
    """(3, n) positions in [0, L): a random subset of a simple-cubic lattice with at least n
    sites, each site displaced by Gaussian noise of width sigma and folded into the box.
    Nearest distances are about L / ceil(n^(1/3)) - a few sigma, as in a dense liquid."""
    rng = np.random.default_rng(seed)
    k = int(np.ceil(n ** (1.0 / 3.0) - 1e-9))
    while k ** 3 < n:
        k += 1
    a = L / k
    sites = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), -1).reshape(-1, 3)
    pick = rng.permutation(len(sites))[:n]
    p = (sites[pick] + 0.5) * a + rng.normal(0.0, sigma, size=(n, 3))
    p = np.mod(p, L)
    p[p >= L] = 0.0
    return np.ascontiguousarray(p.T)


def uniform_positions(n: int, L: float, seed: int) -> np.ndarray:
    """(3, n) positions uniform in [0, L) (overlaps allowed: tests of invariances only)."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.uniform(0.0, L, size=(3, n)))


def uneven_groups():
    """The uneven batch: (N, walkers) groups."""
    return [(128, 2048), (500, 1024), (1000, 512), (1952, 256), (4000, 128)]


def uneven_params(groups, seed: int):
    """Per-walker (n, rho, b) for a batch of groups: rho ~ U[0.0197, 0.0262] A^-3,
    b ~ U[2.9, 3.2] A, as in the uneven-batch workload."""
    rng = np.random.default_rng(seed)
    out = []
    for n, w in groups:
        rho = rng.uniform(0.0197, 0.0262, size=w)
        b = rng.uniform(2.9, 3.2, size=w)
        out += [(int(n), float(r), float(bb)) for r, bb in zip(rho, b)]
    return out


def pad4(n: int) -> int:
    return (n + 3) // 4 * 4
