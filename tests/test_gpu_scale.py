"""Rings beyond the oracle's reach on the GPU: the paper's counts of real stationary
points for N = 11 and 13 at alpha = 0.75 (1,048,576 and 16,777,216 paths), and the
N = 12, sigma = 1 workload (4,194,304 paths) checked by properties that hold at any size."""
import os

import numpy as np
import pytest

from gpu_common import nphc
from oracle_cases import load_counts
from paper_1104_5497_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N", [11, 13])
def test_paper_counts_large_rings(N):
    N_ = nphc()
    counts = load_counts(os.path.join(GOLDEN, "paper_sp_counts.txt"))
    inst = I.paper_ring(N)
    system = N_.System(N, inst.sigma)
    res = N_.solve(system, N_.options_default(gamma=inst.gamma))
    c = res.counts()
    assert c["paths"] == 4 ** (N - 1)
    assert c["real"] == counts[N], (c["real"], counts[N])
    assert c["duplicate"] == 0, (c["duplicate"], c["undecided"], c["handoff"], c["retracked"])
    assert c["index_hist"][0] == 1   # one minimum (the ferromagnetic state)


def test_n12_workload_properties():
    """N = 12, sigma = 1: every path ends in a final status; the real SPs are closed under
    theta -> -theta and under the ring reflection k -> N - k (circulant J); the ground
    state has V = 0 and index 0; no certified solution twice."""
    N_ = nphc()
    inst = I.workload_n12()
    N, M = inst.N, inst.N - 1
    system = N_.System(N, inst.sigma)
    res = N_.solve(system, N_.options_default(gamma=inst.gamma))
    c = res.counts()
    assert c["paths"] == 4 ** M
    assert c["reached"] + c["diverged"] + c["failed"] == c["paths"]
    assert c["duplicate"] == 0
    sps = res.stationary_points()
    th = sps["theta"]
    assert len(th) == c["real"] > 0
    # theta -> -theta and the reflection theta_k -> theta_{N-k} (theta_N = 0 pinned):
    # nearest neighbours on the embedding (cos theta, sin theta)
    from scipy.spatial import cKDTree
    emb = lambda a: np.concatenate([np.cos(a), np.sin(a)], axis=1)
    tree = cKDTree(emb(th))
    for img in (-th, th[:, ::-1], -th[:, ::-1]):
        d, _ = tree.query(emb(img), k=1)
        assert d.max() < 1e-8
    assert np.sum(sps["index"] == 0) == 1
    k = int(np.argmin(sps["energy"]))
    assert abs(sps["energy"][k]) < 1e-12 and sps["index"][k] == 0
