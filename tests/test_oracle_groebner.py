"""The number of finite solutions, pinned by exact algebra: for rings with rational
couplings the stationary equations (section "A First Application", theta_N = 0) are
rebuilt here from their definition over the rationals, and the dimension of the
quotient ring by their Groebner basis (grevlex) counts the complex solutions with
multiplicity.  The oracle must certify exactly that many (real + non-real), none
singular: every solution is then simple and found, and the count of non-real solutions,
which the paper does not print, is fixed independently of any homotopy."""
import numpy as np
import pytest

import oracle as O

sp = pytest.importorskip("sympy")


def xy_polys(N, J):
    m = N - 1
    c = sp.symbols(f"c0:{m}")
    s = sp.symbols(f"s0:{m}")
    eqs = []
    for k in range(m):
        f = 0
        for j in range(N):
            if j == k:
                continue
            cj = 1 if j == N - 1 else c[j]     # theta_N = 0: c_N = 1, s_N = 0
            sj = 0 if j == N - 1 else s[j]
            f += sp.sympify(J[k][j]) * (s[k] * cj - sj * c[k])   # exact: int or Rational
        eqs.append(sp.expand(f))
    eqs += [c[k] ** 2 + s[k] ** 2 - 1 for k in range(m)]
    return eqs, list(c) + list(s)


def quotient_dim(eqs, vs):
    G = sp.groebner(eqs, *vs, order="grevlex")
    assert G.is_zero_dimensional
    lead = [sp.Poly(g, *vs).monoms(order="grevlex")[0] for g in G.exprs]
    n = len(vs)

    def standard(mono):
        return not any(all(mono[i] >= l[i] for i in range(n)) for l in lead)

    seen, todo = set(), [(0,) * n]
    while todo:
        mono = todo.pop()
        if mono in seen or not standard(mono):
            continue
        seen.add(mono)
        todo += [mono[:i] + (mono[i] + 1,) + mono[i + 1:] for i in range(n)]
    return len(seen)


def integer_couplings(N, seed):
    rng = np.random.default_rng(seed)
    J = np.zeros((N, N), dtype=int)
    for i in range(N):
        for j in range(i + 1, N):
            J[i, j] = J[j, i] = int(rng.integers(1, 9))
    return J


CASES = [(3, np.ones((3, 3), int) - np.eye(3, dtype=int)), (3, np.array([[0, 2, 3], [2, 0, 5], [3, 5, 0]]))]
CASES += [(4, integer_couplings(4, seed)) for seed in (0, 1, 2)]


def check(N, J):
    d = quotient_dim(*xy_polys(N, J.tolist()))
    out = O.solve_system(O.xy_terms(N, J.astype(float)), np.exp(0.5j))
    cls = out["cls"]
    assert (cls == O.C_SINGULAR).sum() == 0 and (cls == O.C_UNDECIDED).sum() == 0
    assert ((cls == O.C_REAL) | (cls == O.C_NONREAL)).sum() == d, (N, d, np.bincount(cls))
    return d


@pytest.mark.parametrize("case", range(len(CASES)))
def test_certified_count_equals_groebner_count(case):
    N, J = CASES[case]
    check(N, J)


def ring_couplings(N):
    """J_ij = d_ij^-sigma at sigma = 1 (exact rationals 1/d)."""
    return [[0 if i == j else sp.Rational(1, min(abs(i - j), N - abs(i - j))) for j in range(N)]
            for i in range(N)]


def test_uniform_ring_n4_has_a_positive_dimensional_solution_set():
    """The power-law ring with N = 4 (sigma = 1): the ideal is not zero-dimensional, i.e.
    pinning theta_N leaves a continuum of solutions; the reading that such endpoints are
    singular, counted but never certified, rests on this."""
    eqs, vs = xy_polys(4, ring_couplings(4))
    assert not sp.groebner(eqs, *vs, order="grevlex").is_zero_dimensional


@pytest.mark.slow
def test_uniform_ring_n5_count_equals_groebner_count():
    """The power-law ring with N = 5 at sigma = 1 (8 unknowns, 256 paths; ~30 s of exact
    algebra): the oracle certifies as many solutions as the quotient ring's dimension."""
    d = quotient_dim(*xy_polys(5, ring_couplings(5)))
    out = O.solve_xy(5, 1.0, np.exp(0.5j))
    cls = out["cls"]
    assert (cls == O.C_SINGULAR).sum() == 0 and (cls == O.C_UNDECIDED).sum() == 0
    assert ((cls == O.C_REAL) | (cls == O.C_NONREAL)).sum() == d


# Rings with one coupling shrunk to 2^-e (exactly representable, so the oracle sees the
# same rational system): at J_12 = 0 a pair of solutions sits at infinity, and just
# beside it the pair is finite with a norm ~1 / J_12 (1.6e4 .. 8.4e6 here).  These pin
# the reading of what "goes to infinity" means: every isolated solution is found, however
# large, when a path counts as diverging only once ||z||_inf exceeds 1e8, and the
# singularity test scales with ||z||_inf^2 (an isolated solution of norm 1e6 has a
# Jacobian condition number ~1e12).
def far_case(N, seed, i, j, e):
    if seed is None:
        Ji = np.ones((N, N), int) - np.eye(N, dtype=int)
    else:
        Ji = integer_couplings(N, seed)
    Jr = [[sp.Integer(int(v)) for v in row] for row in Ji]
    Jr[i][j] = Jr[j][i] = sp.Rational(1, 2 ** e)
    J = Ji.astype(float)
    J[i, j] = J[j, i] = 2.0 ** -e
    return Jr, J


FAR_CASES = [(3, None, 0, 1, 15), (3, None, 0, 1, 24), (4, 0, 0, 1, 16), (4, 1, 0, 1, 16),
             (4, 2, 1, 2, 16)]


@pytest.mark.parametrize("case", FAR_CASES)
def test_far_solutions_certified_count_equals_groebner_count(case):
    N = case[0]
    Jr, J = far_case(*case)
    d = quotient_dim(*xy_polys(N, Jr))
    T = O.xy_terms(N, J)
    out = O.solve_system(T, np.exp(0.5j))
    cls = out["cls"]
    cert = (cls == O.C_REAL) | (cls == O.C_NONREAL)
    assert (cls == O.C_SINGULAR).sum() == 0 and (cls == O.C_UNDECIDED).sum() == 0
    assert cert.sum() == d, (d, np.bincount(cls))
    assert np.abs(out["z"][cert]).max() > 1e4   # the case reaches beyond the old radius
    # the reading this replaces (a radius of 1e4) misses the far pair
    short = O.solve_system(T, np.exp(0.5j), track_opts=O.default_track_opts(r_div=1e4))
    assert ((short["cls"] == O.C_REAL) | (short["cls"] == O.C_NONREAL)).sum() < d
