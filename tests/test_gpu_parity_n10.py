"""Full-size parity: the N=10 workload (262,144 paths, the benchmark's configuration and
launch) in both precisions against the oracle.  The certified real and non-real sets
must be identical and every real stationary point must carry the oracle's angles,
Hessian index and energy."""
from functools import lru_cache

import numpy as np
import pytest

import oracle as O
from gpu_common import nphc, torus_dist
from paper_1104_5497_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@lru_cache(maxsize=None)
def oracle_n10():
    inst = I.workload_n10()
    return O.solve_xy(inst.N, inst.sigma, inst.gamma)


def nearest_rel(za, zb):
    """For every point of za, the distance to its nearest point of zb relative to
    1 + |z| (k-d tree on the real embedding), and that point's index."""
    from scipy.spatial import cKDTree
    emb = lambda z: np.concatenate([z.real, z.imag], axis=1)
    d, j = cKDTree(emb(zb)).query(emb(za), k=1)
    return d / (1 + np.linalg.norm(za, axis=1)), j


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_parity_n10_workload(prec):
    N_ = nphc()
    inst = I.workload_n10()
    ref = oracle_n10()
    system = N_.System(inst.N, inst.sigma)
    p = N_.PREC_MIXED if prec == "mixed" else N_.PREC_FP64
    res = N_.solve(system, N_.options_default(gamma=inst.gamma, precision=p))
    ep, sps, counts = res.endpoints(), res.stationary_points(), res.counts()
    assert counts["paths"] == 4 ** (inst.N - 1)
    for cl_gpu, cl_or in ((N_.END_REAL, O.C_REAL), (N_.END_NONREAL, O.C_NONREAL)):
        za = ep["z"][ep["cls"] == cl_gpu]
        zb = ref["z"][ref["cls"] == cl_or]
        assert len(za) == len(zb), (cl_gpu, len(za), len(zb))
        d, j = nearest_rel(zb, za)   # one to one: distinct partners within 1e-10
        assert d.max() <= 1e-10
        assert len(np.unique(j)) == len(zb)
    assert counts["duplicate"] == 0
    ref_th = np.array([s["theta"] for s in ref["sps"]]).reshape(len(ref["sps"]), inst.N - 1)
    assert len(sps["theta"]) == len(ref_th) == counts["real"]
    for th, ix, en in zip(sps["theta"], sps["index"], sps["energy"]):
        d = torus_dist(ref_th, th)
        k = int(d.argmin())
        assert d[k] < 1e-9
        assert ref["sps"][k]["index"] == ix
        assert abs(ref["sps"][k]["energy"] - en) < 1e-10
    hist = np.bincount([s["index"] for s in ref["sps"]], minlength=inst.N)
    assert counts["index_hist"][:inst.N] == hist.tolist()
    # and the histogram obeys Morse theory on the torus T^(N-1) (test_oracle_morse.py)
    from test_oracle_morse import check_morse
    check_morse(np.array(counts["index_hist"][:inst.N]), inst.N)
