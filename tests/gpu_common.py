"""Helpers for the GPU parity tests: build/load the CUDA library once per session and
compare its results with the oracle's."""
from functools import lru_cache

import numpy as np
import pytest

import oracle as O


@lru_cache(maxsize=None)
def nphc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_5497_gb300 import build
    build.build()
    import paper_1104_5497_gb300.nphc as N
    N.lib()
    return N


@lru_cache(maxsize=None)
def oracle_xy(N, sigma, gamma_re, gamma_im):
    return O.solve_xy(N, sigma, complex(gamma_re, gamma_im))


def torus_dist(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b)))).max(axis=-1)


def certified_set(z, cls, classes):
    return z[np.isin(cls, classes)]


def assert_same_point_sets(za, zb, rel=1e-10):
    """za (GPU) and zb (oracle) are the same set: equal sizes, and every point of zb has
    its nearest point of za within rel (1 + |z|), each point of za the partner of exactly
    one point of zb (a one-to-one matching)."""
    assert len(za) == len(zb), (len(za), len(zb))
    if len(zb) == 0:
        return
    partner = np.empty(len(zb), dtype=np.int64)
    for k, z in enumerate(zb):
        d = np.linalg.norm(za - z, axis=1)
        partner[k] = int(d.argmin())
        assert d[partner[k]] <= rel * (1 + np.linalg.norm(z)), d[partner[k]]
    assert len(np.unique(partner)) == len(zb)


def compare_with_oracle(N, sigma, gamma, prec, ref=None, system=None):
    """Solve on the GPU and check: certified real and non-real sets equal the oracle's
    (within 1e-10 relative, one to one), the real SPs carry the same theta, index and
    energy.  system: a prepared system (e.g. with disordered couplings; ref must then be
    the oracle's solve of the same couplings)."""
    N_ = nphc()
    if system is None:
        system = N_.System(N, sigma)
    res = N_.solve(system, N_.options_default(gamma=gamma, precision=prec))
    ep = res.endpoints()
    sps = res.stationary_points()
    counts = res.counts()
    if ref is None:
        ref = oracle_xy(N, float(sigma), float(np.real(gamma)), float(np.imag(gamma)))
    for cl_gpu, cl_or in ((N_.END_REAL, O.C_REAL), (N_.END_NONREAL, O.C_NONREAL)):
        assert_same_point_sets(certified_set(ep["z"], ep["cls"], [cl_gpu]),
                               certified_set(ref["z"], ref["cls"], [cl_or]))
    ref_th = np.array([s["theta"] for s in ref["sps"]]).reshape(len(ref["sps"]), N - 1)
    assert len(ref_th) == len(sps["theta"])
    for th, ix, en, ld in zip(sps["theta"], sps["index"], sps["energy"], sps["log_abs_det"]):
        d = torus_dist(ref_th, th)
        k = int(d.argmin())
        assert d[k] < 1e-9
        assert ref["sps"][k]["index"] == ix
        assert abs(ref["sps"][k]["energy"] - en) < 1e-10
        assert abs(ref["sps"][k]["log_abs_det"] - ld) < 1e-8 * (1 + abs(ld))
    assert counts["duplicate"] == 0 or prec == N_.PREC_FP64
    return res, counts, ref
