"""Seeded synthetic inputs for the power-law XY workloads.

This module draws random numbers and nothing else: it holds none of the method's
arithmetic (no couplings, no polynomial system, no tracking).  Both the CUDA path and
the CPU oracle take their inputs from here, so that the two sides see exactly the same
instance.  Each side turns the draws into couplings and a polynomial system itself.

An instance is (N, sigma, gamma, g): the ring size, the power-law exponent, the
homotopy constant gamma = exp(i phi) with phi ~ U[0, 2 pi), and an optional symmetric
N x N matrix g of per-pair standard normal draws (zero diagonal) for the disordered
couplings J_ij = d_ij^-sigma (1 + 0.1 g_ij).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Instance:
    N: int
    sigma: float
    gamma: complex
    g: np.ndarray | None = None   # symmetric per-pair draws, or None for the clean ring
    eps: float = 0.1              # disorder strength multiplying g

    @property
    def n(self) -> int:
        return 2 * (self.N - 1)

    @property
    def npaths(self) -> int:
        return 1 << self.n


def draw_gamma(rng: np.random.Generator) -> complex:
    phi = rng.uniform(0.0, 2.0 * np.pi)
    return complex(np.cos(phi), np.sin(phi))


def draw_pair_normals(rng: np.random.Generator, N: int) -> np.ndarray:
    """One N(0,1) draw per unordered pair i < j, mirrored to keep g symmetric."""
    g = np.zeros((N, N))
    iu = np.triu_indices(N, 1)
    g[iu] = rng.standard_normal(len(iu[0]))
    return g + g.T


def ring(N: int, sigma: float, seed: int) -> Instance:
    """Clean power-law ring with a seeded gamma."""
    rng = np.random.default_rng(seed)
    return Instance(N=N, sigma=float(sigma), gamma=draw_gamma(rng))


def ring_random_sigma(N: int, seed: int, lo: float = 0.5, hi: float = 3.0) -> Instance:
    """Clean ring with sigma ~ U[lo, hi] and gamma drawn from the same seed."""
    rng = np.random.default_rng(seed)
    sigma = float(rng.uniform(lo, hi))
    return Instance(N=N, sigma=sigma, gamma=draw_gamma(rng))


def disordered_batch(count: int, seed: int, n_lo: int = 6, n_hi: int = 9,
                     s_lo: float = 0.5, s_hi: float = 3.0) -> list[Instance]:
    """A batch of disordered rings: N ~ U{n_lo..n_hi}, sigma ~ U[s_lo, s_hi], one g per pair."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(n_lo, n_hi + 1))
        sigma = float(rng.uniform(s_lo, s_hi))
        gamma = draw_gamma(rng)
        g = draw_pair_normals(rng, N)
        out.append(Instance(N=N, sigma=sigma, gamma=gamma, g=g))
    return out


# The five workloads the library is measured and tested on, named by what they are.
def workload_n4() -> Instance:
    """N=4, sigma=1.5: 6 unknowns, 64 paths."""
    return ring(4, 1.5, seed=0)


def workload_n8() -> Instance:
    """N=8, sigma=1.5: 14 unknowns, 16,384 paths."""
    return ring(8, 1.5, seed=1)


def workload_n10() -> Instance:
    """N=10, sigma ~ U[0.5, 3]: 18 unknowns, 262,144 paths."""
    return ring_random_sigma(10, seed=2)


def workload_batch64() -> list[Instance]:
    """64 disordered rings with N in 6..9: 1,024 to 65,536 paths each."""
    return disordered_batch(64, seed=3)


def workload_n12() -> Instance:
    """N=12, sigma=1.0: 22 unknowns, 4,194,304 paths."""
    return ring(12, 1.0, seed=4)


def paper_ring(N: int, seed: int = 5) -> Instance:
    """The paper's replication runs: alpha = sigma = 0.75 (odd N = 3..13)."""
    return ring(N, 0.75, seed=seed + N)
