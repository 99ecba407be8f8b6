"""Pins for the oracle's Cauchy endgame (oracle_endgame): systems whose singular endpoints,
cycle numbers and paths to infinity are known in closed form, nonsingular endpoints
against the known roots, and the singular endpoints of the N = 0 mod 4 rings against the
definition of a solution (P(z) = 0)."""
import numpy as np
import pytest

import oracle as O
import systems as S

GAMMA = np.exp(0.5j)


def run(T, paths=None, **kw):
    paths = np.arange(2 ** T.n) if paths is None else paths
    return O.endgame(T, GAMMA, paths, eg_opts=O.default_eg_opts(**kw))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_squares_end_at_zero_with_cycle_two(n):
    r = run(S.squares(n))
    assert np.all(r["status"] == O.EG_CONVERGED)
    assert np.all(r["cycle"] == 2)
    assert np.abs(r["z"]).max() < 1e-12


def test_one_turn_never_closes_on_a_cycle_two_path():
    """z_i ~ +-sqrt(gamma (1-t)) near t = 1: one turn around t = 1 takes each sheet to the
    other, so with max_cycle = 1 no radius closes; with 2 every path closes after two."""
    r = run(S.squares(2), max_cycle=1)
    assert np.all(r["status"] == O.EG_NOT_CLOSED)
    assert np.all(r["cycle"] == 0)
    r2 = run(S.squares(2), max_cycle=2)
    assert np.all(r2["status"] == O.EG_CONVERGED) and np.all(r2["cycle"] == 2)


def test_double_root_estimates_and_multiplicity():
    a, b = 0.3 + 0.2j, 2.0
    r = run(S.double_root(a, b))
    assert np.all(r["status"] == O.EG_CONVERGED)
    assert np.all(r["cycle"] == 2)
    assert np.abs(r["z"][:, 0] - a).max() < 1e-12
    z2 = r["z"][:, 1]
    assert np.abs(np.abs(z2) - np.sqrt(b)).max() < 1e-12
    # each of +-sqrt(b) is the end of two paths (z_2 is nonsingular; z_1 is the double root)
    assert sorted(np.sign(z2.real).tolist()) == [-1, -1, 1, 1]


def test_chain_has_cycle_four():
    r = run(S.chain4())
    assert np.all(r["status"] == O.EG_CONVERGED)
    assert np.all(r["cycle"] == 4)
    assert np.abs(r["z"]).max() < 1e-12
    # cycle numbers above max_cycle are not found at any radius
    r3 = run(S.chain4(), max_cycle=3)
    assert np.all(r3["status"] == O.EG_NOT_CLOSED)


@pytest.mark.parametrize("seed", [1, 2])
def test_nonsingular_endpoints_have_cycle_one_and_match_the_roots(seed):
    T, roots = S.product_system(3, seed)
    r = run(T)
    assert np.all(r["status"] == O.EG_CONVERGED)
    assert np.all(r["cycle"] == 1)
    for z in r["z"]:
        d = np.linalg.norm(roots - z, axis=1)
        assert d.min() < 1e-11 * (1 + np.linalg.norm(z))
    r5 = run(S.x2_minus_5())
    assert np.allclose(np.sort(r5["z"][:, 0].real), [-np.sqrt(5), np.sqrt(5)], atol=1e-13)


def test_paths_to_infinity():
    """P = z - 2 tracked from z^2 - 1: one path ends at 2, the other goes to infinity as
    -t / (gamma (1 - t)); z_1 z_2 = 1, z_2^2 = z_2: the solution (1, 1) and three paths to
    infinity (z_2 -> 0 forces z_1 -> infinity)."""
    r = run(O.Terms(1, [0, 0], [0, -1], [-1, -1], [1.0, -2.0]))
    assert r["status"].tolist() == [O.EG_CONVERGED, O.EG_AT_INFINITY]
    assert abs(r["z"][0, 0] - 2) < 1e-13
    T2 = O.Terms(2, [0, 0, 1, 1], [0, -1, 1, 1], [1, -1, 1, -1], [1.0, -1.0, 1.0, -1.0])
    r2 = run(T2)
    ok = r2["status"] == O.EG_CONVERGED
    assert ok.sum() == 1 and np.abs(r2["z"][ok][0] - [1, 1]).max() < 1e-13
    assert np.all(r2["status"][~ok] == O.EG_AT_INFINITY)


def test_wrong_radius_schedule_is_caught_by_agreement():
    """With one radius there is nothing to compare: the estimate is returned as not
    converged (and is still the endpoint for a clean path)."""
    r = run(S.double_root(0.3 + 0.2j, 2.0), n_radii=1)
    assert np.all(r["status"] == O.EG_NOT_CONVERGED)
    assert np.abs(r["z"][:, 0] - (0.3 + 0.2j)).max() < 1e-10


@pytest.mark.parametrize("N", [4, 8])
def test_ring_singular_endpoints_are_solutions(N):
    """Rings with N = 0 mod 4 have positive-dimensional solution sets: paths that end there
    do not certify.  The endgame reaches them: every converged estimate solves P to
    rounding, with a cycle number >= 2 (several paths meet there); every path that the
    tracker left singular converges; the others go to infinity.  A slow path to infinity
    that stalled below the divergence radius (1e8) may stay undecided after the last
    radius (its turn means agree only to ~1e-8); its estimate then does not solve P."""
    out = O.solve_xy(N, 1.0, GAMMA)
    sel = np.nonzero(np.isin(out["cls"], [O.C_SINGULAR, O.C_FAILED]))[0]
    assert len(sel) > 0
    T = O.xy_terms(N, out["J"])
    r = O.endgame(T, GAMMA, out["path"][sel])
    ok = r["status"] == O.EG_CONVERGED
    undecided = r["status"] == O.EG_NOT_CONVERGED
    assert np.all(ok | undecided | (r["status"] == O.EG_AT_INFINITY))
    assert np.all(ok[out["cls"][sel] == O.C_SINGULAR])
    for z in r["z"][undecided]:
        scale = max(1.0, np.abs(z).max() ** 2)
        assert np.abs(T.eval_acc(z)).max() > 1e3 * 1e-10 * scale
    for z in r["z"][ok]:
        assert np.abs(T.eval_acc(z)).max() < 1e-12
    assert np.all(r["cycle"][ok] >= 2)
    # a real endpoint on the constraint circles: c_k^2 + s_k^2 = 1
    m = N - 1
    zr = r["z"][ok]
    assert np.abs(zr[:, :m] ** 2 + zr[:, m:] ** 2 - 1).max() < 1e-12


def test_trapezoid_estimate_matches_closed_form():
    """K = 2 samples per turn at the single radius r = 1/2 (no other branch point inside:
    the discriminant's other zero and the poles lie beyond |1 - t| = 1.5).  For the double
    root (z_1 - a)^2 the turns close after two turns and visit both roots at t = 1 - r
    (theta = 0, 2 pi) and at t = 1 + r (theta = pi, 3 pi); by Vieta the two roots of
    (gamma (1-t) + t) z^2 - 2 t a z + ... sum to 2 f(t), f(t) = t a / (gamma (1-t) + t), so
    the estimate of z_1 is (f(1 - r) + f(1 + r)) / 2.  z_2 = +-sqrt(g(t)), g(t) = (gamma (1-t)
    + t b) / (gamma (1-t) + t), is analytic inside the circle: its estimate is the mean of
    the branch at 1 - r and at 1 + r, continued along real t."""
    a, b, r = 0.3 + 0.2j, 2.0, 0.5
    f = lambda t: t * a / (GAMMA * (1 - t) + t)
    g = lambda t: (GAMMA * (1 - t) + t * b) / (GAMMA * (1 - t) + t)
    T = S.double_root(a, b)
    res = run(T, r0=r, n_radii=1, samples=2)
    assert np.all(res["status"] == O.EG_NOT_CONVERGED) and np.all(res["cycle"] == 2)
    assert np.abs(res["z"][:, 0] - (f(1 - r) + f(1 + r)) / 2).max() < 1e-11
    ts = np.linspace(1 - r, 1 + r, 20001)
    for p in range(4):
        # the branch of z_2 along real t through t = 1, from the path's sign at t = 1 - r
        w = np.sqrt(g(ts))
        for k in range(1, len(ts)):
            if abs(w[k] - w[k - 1]) > abs(w[k] + w[k - 1]):
                w[k:] = -w[k:]
        z_end = O.track(T, GAMMA, path0=p, npaths=1)["z"][0, 1]   # the path's z_2 at t = 1
        mid = len(ts) // 2                                          # ts[mid] = 1
        sgn = np.sign((w[mid] * np.conj(z_end)).real)
        expect = sgn * (w[0] + w[-1]) / 2
        assert abs(res["z"][p, 1] - expect) < 1e-10, (p, res["z"][p, 1], expect)
