"""GPU vs oracle parity of the whole method (track, refine, certify, dedup, classify)
through the C ABI: the certified solution sets must be identical and every real
stationary point must carry the same angles, Hessian index and energy."""
import os

import numpy as np
import pytest

import oracle as O
from gpu_common import compare_with_oracle, nphc
from oracle_cases import load_counts
from paper_1104_5497_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("N,sigma,seed", [(3, 0.75, 5), (4, 1.5, 0), (5, 0.75, 10), (6, 1.5, 3),
                                          (7, 0.75, 12), (7, 2.5, 4)])
def test_parity_small_rings(N, sigma, seed, prec):
    N_ = nphc()
    inst = I.ring(N, sigma, seed)
    p = N_.PREC_MIXED if prec == "mixed" else N_.PREC_FP64
    compare_with_oracle(N, sigma, inst.gamma, p)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_parity_n8_workload(prec):
    """The N=8, sigma=1.5 workload: 16,384 paths, positive-dimensional real families
    (N = 0 mod 4) whose singular endpoints must not certify."""
    N_ = nphc()
    inst = I.workload_n8()
    p = N_.PREC_MIXED if prec == "mixed" else N_.PREC_FP64
    res, counts, ref = compare_with_oracle(inst.N, inst.sigma, inst.gamma, p)
    assert counts["paths"] == 4 ** (inst.N - 1)


def test_paper_counts_on_gpu():
    """N = 3, 5, 7, 9 at alpha = 0.75: 6, 20, 168, 972 real stationary points."""
    N_ = nphc()
    counts = load_counts(os.path.join(GOLDEN, "paper_sp_counts.txt"))
    for N in (3, 5, 7, 9):
        inst = I.paper_ring(N)
        system = N_.System(N, inst.sigma)
        res = N_.solve(system, N_.options_default(gamma=inst.gamma))
        c = res.counts()
        assert c["real"] == counts[N], (N, c)
        assert c["duplicate"] == 0


def test_disordered_ring():
    """A disordered ring of the 64-instance batch workload (J scaled per pair)."""
    N_ = nphc()
    inst = I.disordered_batch(4, seed=3)[1]
    J = N_.xy_couplings(inst.N, inst.sigma, inst.g, inst.eps)
    Jo = O.couplings(inst.N, inst.sigma, inst.g, inst.eps)
    assert np.array_equal(J, Jo)
    system = N_.System(inst.N, inst.sigma, J)
    res = N_.solve(system, N_.options_default(gamma=inst.gamma))
    ref = O.solve_xy(inst.N, inst.sigma, inst.gamma, g=inst.g, eps=inst.eps)
    c = res.counts()
    assert c["real"] == (ref["cls"] == O.C_REAL).sum()
    assert c["nonreal"] == (ref["cls"] == O.C_NONREAL).sum()


def test_disordered_n9_ring_point_sets():
    """An N = 9 ring of the 64-instance batch workload (per-pair disorder, 65,536 paths) in
    mixed precision: the certified real and non-real sets are the oracle's one to one, and
    every real SP has the oracle's angles, index and energy."""
    N_ = nphc()
    inst = I.workload_batch64()[0]
    assert inst.N == 9
    J = N_.xy_couplings(inst.N, inst.sigma, inst.g, inst.eps)
    system = N_.System(inst.N, inst.sigma, J)
    ref = O.solve_xy(inst.N, inst.sigma, inst.gamma, g=inst.g, eps=inst.eps)
    compare_with_oracle(inst.N, inst.sigma, inst.gamma, N_.PREC_MIXED, ref=ref, system=system)
