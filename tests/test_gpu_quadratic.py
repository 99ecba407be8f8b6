"""Generic quadratic systems on the GPU (nphc_system_create_quadratic) against the paper's
worked example, closed-form roots and the oracle."""
import math
import os

import numpy as np
import pytest

import oracle as O
from gpu_common import nphc
from systems import product_system, random_quadratic, x2_minus_5

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gpu_system(N_, T):
    return N_.System.quadratic(T.n, T.eq, T.va, T.vb, T.cre + 1j * T.cim)


def gpu_solve(N_, T, gamma):
    system = gpu_system(N_, T)
    res = N_.solve(system, N_.options_default(gamma=gamma))
    return system, res, res.endpoints(), res.counts()


def match(za, zb, rel=1e-10):
    """Every point of za has a partner in zb (and the sets have the same size)."""
    assert len(za) == len(zb), (len(za), len(zb))
    for z in za:
        d = np.linalg.norm(zb - z, axis=1)
        assert d.min() <= rel * (1 + np.linalg.norm(z)), d.min()


@pytest.mark.parametrize("phi", [0.3, 1.9, 4.4])
def test_paper_worked_example_x2_minus_5(phi):
    """x^2 - 5 tracked from x^2 - 1: the start points +1 and -1 end at +sqrt 5 and
    -sqrt 5, both certified real; the paper prints 2.236067977."""
    N_ = nphc()
    printed, prec = [float(v) for v in open(os.path.join(GOLDEN, "x2_minus_5.txt"))
                     .read().split("\n")[-2].split()]
    system, res, ep, c = gpu_solve(N_, x2_minus_5(), complex(math.cos(phi), math.sin(phi)))
    assert system.N == 0 and system.n == 1 and system.npaths == 2
    assert list(ep["status"]) == [N_.PATH_REACHED, N_.PATH_REACHED]
    assert list(ep["cls"]) == [N_.END_REAL, N_.END_REAL]
    assert abs(ep["z"][0, 0] - math.sqrt(5)) < 1e-14
    assert abs(ep["z"][1, 0] + math.sqrt(5)) < 1e-14
    assert abs(ep["z"][0, 0].real - printed) < prec
    assert c["real"] == 2 and c["duplicate"] == 0


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2), (5, 3), (7, 5)])
def test_product_system_all_roots(n, seed):
    """(w_i - a_i)(w_i - b_i) with w = A z: all 2^n roots, each once, certified, with the
    real ones (a_i, b_i real) certified real."""
    N_ = nphc()
    T, roots = product_system(n, seed)
    system, res, ep, c = gpu_solve(N_, T, np.exp(1j * 2.1))
    cert = np.isin(ep["cls"], [N_.END_REAL, N_.END_NONREAL, N_.END_UNDECIDED])
    assert cert.sum() == 2 ** n and c["duplicate"] == 0
    match(ep["z"][cert], roots)
    real = np.all(np.abs(roots.imag) < 1e-12, axis=1)
    assert c["real"] == real.sum()


@pytest.mark.parametrize("n,seed,density", [(3, 11, 1.0), (4, 12, 1.0), (6, 13, 0.5),
                                            (8, 14, 0.3)])
def test_random_quadratic_matches_oracle(n, seed, density):
    """Random complex quadratic systems: the GPU's certified set, classes and the count
    of each class equal the oracle's."""
    N_ = nphc()
    T = random_quadratic(n, seed, density)
    gamma = np.exp(1j * 0.7)
    ref = O.solve_system(T, gamma)
    system, res, ep, c = gpu_solve(N_, T, gamma)
    for cg, co in ((N_.END_REAL, O.C_REAL), (N_.END_NONREAL, O.C_NONREAL),
                   (N_.END_UNDECIDED, O.C_UNDECIDED)):
        match(ep["z"][ep["cls"] == cg], ref["z"][ref["cls"] == co])


def test_quadratic_step_by_step_matches_oracle_per_path():
    """nphc_track + nphc_refine_certify on a quadratic system: every path the oracle
    certifies ends, on the GPU, at the same solution (paths are unique)."""
    import torch
    N_ = nphc()
    T = random_quadratic(5, 21)
    gamma = np.exp(1j * 2.5)
    ref = O.solve_system(T, gamma)
    system = gpu_system(N_, T)
    P = system.npaths
    ep = N_.DeviceEndpoints.empty(T.n, np.arange(P))
    ws = torch.zeros(system.workspace_size(P), dtype=torch.uint8, device="cuda")
    opts = N_.options_default(gamma=gamma)
    N_.track(system, opts, N_.PREC_FP64, ep, ws)
    N_.refine_certify(system, opts, ep)
    torch.cuda.synchronize()
    cls = ep.tensors["cls"].cpu().numpy()
    z = ep.tensors["z_re"].cpu().numpy().T + 1j * ep.tensors["z_im"].cpu().numpy().T
    cert = np.isin(ref["cls"], [O.C_REAL, O.C_NONREAL])
    assert np.array_equal(np.isin(cls, [N_.END_REAL, N_.END_NONREAL]), cert)
    d = np.linalg.norm(z[cert] - ref["z"][cert], axis=1)
    assert (d <= 1e-10 * (1 + np.linalg.norm(ref["z"][cert], axis=1))).all()


def test_quadratic_system_rejects_classification():
    import torch
    N_ = nphc()
    system = gpu_system(N_, x2_minus_5())
    res = N_.solve(system, N_.options_default())
    with pytest.raises(N_.NphcError):
        res.stationary_points()
    ep = N_.DeviceEndpoints.empty(1, np.arange(2))
    th = torch.zeros(1, 2, dtype=torch.float64, device="cuda")
    ix = torch.zeros(2, dtype=torch.int32, device="cuda")
    en = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(N_.NphcError):
        N_.classify(system, ep, th, ix, en)
