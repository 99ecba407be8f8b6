"""The Cauchy endgame on the GPU (nphc_endgame, cauchy.cuh) against the oracle's
(oracle_endgame) on the same paths: the same outcome and cycle number per path, endpoint
estimates within 1e-8 (relative).  Cases: the closed-form systems of tests/systems.py
(singular endpoints with cycle numbers 2 and 4, paths to infinity, a near double root
whose branch point lies inside the first radii), the paths of the N = 4 and N = 8 rings
that end singular or fail (positive-dimensional solution sets), and the pipeline option
opts.endgame on the N = 8 ring."""
import numpy as np
import pytest

import oracle as O
import systems as S
from gpu_common import nphc

pytestmark = pytest.mark.gpu
GAMMA = np.exp(0.5j)


def gpu_endgame(N_, system, paths, **kw):
    import torch
    opts = N_.options_default(gamma=GAMMA, **kw)
    ep = N_.DeviceEndpoints.empty(system.n, np.asarray(paths, dtype=np.int64))
    ws = torch.empty(system.workspace_size(ep.count), dtype=torch.uint8, device="cuda")
    cyc = torch.zeros(ep.count, dtype=torch.int32, device="cuda")
    st = torch.zeros(ep.count, dtype=torch.int32, device="cuda")
    N_.endgame(system, opts, ep, ws, cyc, st)
    torch.cuda.synchronize()
    z = (ep.tensors["z_re"] + 1j * ep.tensors["z_im"]).T.cpu().numpy()
    return dict(z=z, status=st.cpu().numpy(), cycle=cyc.cpu().numpy())


def compare(g, o, rel=1e-8):
    assert np.array_equal(g["status"], o["status"]), (g["status"], o["status"])
    assert np.array_equal(g["cycle"], o["cycle"]), (g["cycle"], o["cycle"])
    conv = o["status"] == O.EG_CONVERGED
    if conv.any():
        err = np.abs(g["z"][conv] - o["z"][conv]).max(axis=1)
        scale = 1 + np.abs(o["z"][conv]).max(axis=1)
        assert np.all(err <= rel * scale), err.max()


def quad(N_, T):
    return N_.System.quadratic(T.n, T.eq, T.va, T.vb, T.cre + 1j * T.cim)


CLOSED = {
    "squares2": lambda: S.squares(2),
    "squares3": lambda: S.squares(3),
    "double_root": lambda: S.double_root(0.3 + 0.2j, 2.0),
    "chain4": S.chain4,
    "x2_minus_5": S.x2_minus_5,
    "linear": lambda: O.Terms(1, [0, 0], [0, -1], [-1, -1], [1.0, -2.0]),
    "infinity2": lambda: O.Terms(2, [0, 0, 1, 1], [0, -1, 1, 1], [1, -1, 1, -1],
                                 [1.0, -1.0, 1.0, -1.0]),
    "near_double": lambda: S.product_system(3, 1)[0],
    "random4": lambda: S.random_quadratic(4, 3),
}


@pytest.mark.parametrize("name", sorted(CLOSED))
def test_quadratic_systems_match_oracle(name):
    N_ = nphc()
    T = CLOSED[name]()
    paths = np.arange(2 ** T.n)
    o = O.endgame(T, GAMMA, paths)
    g = gpu_endgame(N_, quad(N_, T), paths)
    compare(g, o)


def test_closed_form_values_on_gpu():
    """Independently of the oracle: cycle 2 / 4 and the exact singular endpoints."""
    N_ = nphc()
    g = gpu_endgame(N_, quad(N_, S.chain4()), np.arange(4))
    assert np.all(g["status"] == O.EG_CONVERGED) and np.all(g["cycle"] == 4)
    assert np.abs(g["z"]).max() < 1e-12
    a = 0.3 + 0.2j
    g = gpu_endgame(N_, quad(N_, S.double_root(a, 2.0)), np.arange(4))
    assert np.all(g["cycle"] == 2)
    assert np.abs(g["z"][:, 0] - a).max() < 1e-12
    assert np.abs(np.abs(g["z"][:, 1]) - np.sqrt(2.0)).max() < 1e-12


@pytest.mark.parametrize("N", [4, 8])
def test_ring_singular_and_failed_paths_match_oracle(N):
    N_ = nphc()
    out = O.solve_xy(N, 1.0, GAMMA)
    sel = np.nonzero(np.isin(out["cls"], [O.C_SINGULAR, O.C_FAILED]))[0]
    paths = out["path"][sel]
    o = O.endgame(O.xy_terms(N, out["J"]), GAMMA, paths)
    g = gpu_endgame(N_, N_.System(N, 1.0), paths)
    compare(g, o)
    # slow paths to infinity that stall below the divergence radius may stay undecided
    # after the last radius; their estimates do not solve P (as in the oracle's test)
    assert np.all(np.isin(g["status"], [O.EG_CONVERGED, O.EG_AT_INFINITY, O.EG_NOT_CONVERGED]))
    T = O.xy_terms(N, out["J"])
    for z in g["z"][g["status"] == O.EG_NOT_CONVERGED]:
        assert np.abs(T.eval_acc(z)).max() > 1e3 * 1e-10 * max(1.0, np.abs(z).max() ** 2)


def test_pipeline_option_on_ring_n8():
    """opts.endgame: the solve runs the endgame on its singular and failed paths; the
    counts, classes and statuses of the solve are those without it; the outcomes are the
    oracle's for the same paths."""
    N_ = nphc()
    system = N_.System(8, 1.0)
    base = N_.solve(system, N_.options_default(gamma=GAMMA))
    res = N_.solve(system, N_.options_default(gamma=GAMMA, endgame=1))
    c0, c1 = base.counts(), res.counts()
    for k in ("paths", "reached", "diverged", "failed", "real", "nonreal", "singular", "duplicate"):
        assert c0[k] == c1[k], k
    assert c0["eg_run"] == 0
    e0, e1 = base.endpoints(), res.endpoints()
    assert np.array_equal(e0["cls"], e1["cls"]) and np.array_equal(e0["status"], e1["status"])
    eg = res.endgame()
    run = eg["status"] != N_.EG_NONE
    assert np.array_equal(run, np.isin(e1["cls"], [N_.END_SINGULAR, N_.END_FAILED]))
    assert c1["eg_run"] == run.sum() == c1["singular"] + c1["failed"]
    paths = np.nonzero(run)[0]
    out = O.solve_xy(8, 1.0, GAMMA)
    o = O.endgame(O.xy_terms(8, out["J"]), GAMMA, paths)
    g = dict(z=e1["z"][paths], status=eg["status"][paths], cycle=eg["cycle"][paths])
    compare(g, o)
    conv = o["status"] == O.EG_CONVERGED
    assert c1["eg_converged"] == conv.sum()
    assert c1["eg_multiple"] == (conv & (o["cycle"] >= 2)).sum()
    assert c1["eg_at_infinity"] == np.isin(o["status"], [O.EG_AT_INFINITY, O.EG_DIVERGED]).sum()


def test_two_sample_trapezoid_value_on_gpu():
    """The closed-form trapezoid value of the double root (see the oracle's pin): K = 2
    samples per turn at the single radius 1/2; the estimate of z_1 is
    (f(1 - r) + f(1 + r)) / 2 with f(t) = t a / (gamma (1 - t) + t)."""
    N_ = nphc()
    a, b, r = 0.3 + 0.2j, 2.0, 0.5
    f = lambda t: t * a / (GAMMA * (1 - t) + t)
    g = gpu_endgame(N_, quad(N_, S.double_root(a, b)), np.arange(4), eg_r0=r, eg_radii=1,
                    eg_samples=2)
    assert np.all(g["status"] == N_.EG_NOT_CONVERGED) and np.all(g["cycle"] == 2)
    assert np.abs(g["z"][:, 0] - (f(1 - r) + f(1 + r)) / 2).max() < 1e-11
