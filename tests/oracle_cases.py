"""Cached oracle runs shared by the CPU tests (each instance is solved once per session)."""
from functools import lru_cache

import numpy as np

import oracle as O
from paper_1104_5497_gb300 import inputs as I


@lru_cache(maxsize=None)
def xy(N: int, sigma: float, seed: int):
    inst = I.ring(N, sigma, seed)
    return O.solve_xy(N, inst.sigma, inst.gamma)


def paper(N: int):
    """The paper's runs, sigma = alpha = 0.75 (same seed as inputs.paper_ring)."""
    return xy(N, 0.75, 5 + N)


def certified(out, classes=(O.C_REAL, O.C_NONREAL, O.C_UNDECIDED)):
    return np.isin(out["cls"], classes)


def real_thetas(out):
    th = np.array([s["theta"] for s in out["sps"]])
    return th.reshape(len(out["sps"]), out["N"] - 1)


def load_counts(path):
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {int(a): int(b) for a, b in rows}
