"""Pins for the oracle's homotopy tracker, refinement, certification and dedup on
systems whose solutions are known in closed form."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from systems import product_system, x2_minus_5

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_worked_example_x2_minus_5():
    """Section 'Numerical Polynomial Homotopy Continuation Method': x^2 - 5 from x^2 - 1
    gives +-sqrt(5); the paper prints +-(2.236067977 + i 1e-10)."""
    printed, prec = [float(v) for v in open(os.path.join(GOLDEN, "x2_minus_5.txt"))
                     .read().split("\n")[-2].split()]
    for phi in (0.3, 1.9, 4.4):
        out = O.solve_system(x2_minus_5(), complex(math.cos(phi), math.sin(phi)))
        assert list(out["status"]) == [O.REACHED, O.REACHED]
        z = np.sort_complex(out["z"][:, 0])
        # start point +1 ends at +sqrt 5 and -1 at -sqrt 5 (the paths are x(t) = +-sqrt(1 + 4t)
        # up to the gamma twist, which cannot swap them because they never meet)
        assert abs(out["z"][0, 0] - math.sqrt(5)) < 1e-12
        assert abs(out["z"][1, 0] + math.sqrt(5)) < 1e-12
        assert abs(abs(z[0].real) - printed) < prec and abs(z[1].real - printed) < prec
        assert list(out["cls"]) == [O.C_REAL, O.C_REAL]
        assert out["n_duplicates"] == 0


def test_alpha_closed_form_univariate():
    """For f = x^2 - 5: beta = |f/f'| = |x^2-5|/|2x|, gamma = |f''/(2 f')| = 1/|2x|,
    so alpha = |x^2 - 5| / (4 |x|^2).  The oracle's bound is exact for n = 1."""
    T = x2_minus_5()
    assert T.d2_norm() == pytest.approx(1.0)
    opts = O.default_cert_opts(refine_iters=0)
    for x in (2.2 + 0.01j, 2.3, -2.0 + 0.3j):
        tr = dict(z=np.array([[x]]), status=np.array([O.REACHED], np.int32), tend=np.ones(1))
        rc = O.refine_certify(T, tr, opts)
        beta = abs(x * x - 5) / abs(2 * x)
        gam = 1 / abs(2 * x)
        assert rc["beta"][0] == pytest.approx(beta, rel=1e-13)
        assert rc["gamma"][0] == pytest.approx(gam, rel=1e-13)
        assert rc["alpha"][0] == pytest.approx(beta * gam, rel=1e-13)


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (4, 2), (5, 3)])
def test_product_system_all_roots(n, seed):
    T, roots = product_system(n, seed)
    out = O.solve_system(T, np.exp(1j * 2.1))
    cert = np.isin(out["cls"], [O.C_REAL, O.C_NONREAL, O.C_UNDECIDED])
    assert cert.sum() == 2 ** n and out["n_duplicates"] == 0
    found = out["z"][cert]
    for r in roots:
        d = np.linalg.norm(found - r, axis=1)
        assert d.min() < 1e-10 * (1 + np.linalg.norm(r))
    # the real test agrees with the construction (w real <=> b_i real for the chosen pair)
    real_roots = sum(np.abs(r.imag).max() < 1e-12 for r in roots)
    assert (out["cls"] == O.C_REAL).sum() == real_roots


def test_dedup_flags_second_copy():
    T, roots = product_system(2, 0)
    z = np.stack([roots[0], roots[1], roots[0] + 1e-13])
    tr = dict(z=z, status=np.full(3, O.REACHED, np.int32), tend=np.ones(3))
    rc = O.refine_certify(T, tr)
    assert O.dedup(2, rc) == 1
    assert rc["cls"][2] == O.C_DUPLICATE and rc["cls"][0] != O.C_DUPLICATE


def test_every_path_gets_a_final_status():
    T, _ = product_system(3, 7)
    out = O.track(T, np.exp(0.4j))
    assert (out["status"] != 0).all() and len(out["status"]) == 8


def exact_eval(T, z):
    """P(z) in exact rational arithmetic on the same doubles."""
    from fractions import Fraction as F
    out = []
    for i in range(T.n):
        re = F(0)
        im = F(0)
        for e, a, b, cr, ci in zip(T.eq, T.va, T.vb, T.cre, T.cim):
            if e != i:
                continue
            wa = (F(1), F(0)) if a < 0 else (F(float(z[a].real)), F(float(z[a].imag)))
            wb = (F(1), F(0)) if b < 0 else (F(float(z[b].real)), F(float(z[b].imag)))
            pr, pi = wa[0] * wb[0] - wa[1] * wb[1], wa[0] * wb[1] + wa[1] * wb[0]
            re += F(float(cr)) * pr - F(float(ci)) * pi
            im += F(float(cr)) * pi + F(float(ci)) * pr
        out.append(complex(float(re), float(im)))
    return np.array(out)


def test_compensated_evaluation_is_correctly_rounded_where_plain_is_not():
    """The refinement's P(z): at a large-norm point the plain double sum loses digits to
    cancellation between ~||z||^2 terms; the compensated sum equals the exact value to
    the last bit or so."""
    N = 6
    J = O.couplings(N, 0.9)
    T = O.xy_terms(N, J)
    rng = np.random.default_rng(5)
    worst_acc = worst_plain = 0.0
    for trial in range(20):
        scale = 10.0 ** rng.uniform(0, 4)
        z = scale * (rng.standard_normal(T.n) + 1j * rng.standard_normal(T.n))
        z[T.n // 2:] = 1j * z[:T.n // 2] * (1 + 1e-9 * rng.standard_normal(T.n // 2))  # near y = i x
        ex = exact_eval(T, z)
        acc = T.eval_acc(z)
        plain, _ = T.eval_jac(z)
        ref = np.abs(ex) + 1e-300
        worst_acc = max(worst_acc, (np.abs(acc - ex) / ref).max())
        worst_plain = max(worst_plain, (np.abs(plain - ex) / ref).max())
    assert worst_acc < 4e-16
    assert worst_plain > 1e3 * worst_acc


def test_step_budget_of_one_stops_every_path():
    """A failure made on the host: a step budget of 1 ends every path with the budget
    status after its first attempt (no path reaches t = 1 in one step from h0 = 0.01)."""
    import numpy as np
    import oracle as O
    T = O.xy_terms(4, O.couplings(4, 1.5))
    tr = O.track(T, np.exp(0.5j), opts=O.default_track_opts(max_steps=1))
    assert np.all(tr["status"] == O.STEP_BUDGET)
    assert np.all(tr["steps"] <= 1)
