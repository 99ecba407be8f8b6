"""Pins for the oracle's adjoint (oracle_xy_adjoint): gradients of losses on a stationary
point with respect to the couplings, against central finite differences in which the
same stationary point is Newton-refined under the perturbed couplings (not re-solved:
a re-solve could pick another stationary point).  The gradient and Hessian of V used
here are written from V's definition, independently of the oracle."""
import numpy as np
import pytest

import oracle as O
from oracle_cases import paper, xy
from sp_newton import energy, refine


@pytest.mark.parametrize("case", ["paper5", "ring6", "disordered7"])
def test_adjoint_matches_finite_differences(case):
    if case == "paper5":
        out, N = paper(5), 5
    elif case == "ring6":
        out, N = xy(6, 1.5, 3), 6
    else:
        rng = np.random.default_rng(4)
        g = rng.standard_normal((7, 7))
        g = np.triu(g, 1) + np.triu(g, 1).T
        out = O.solve_xy(7, 1.2, np.exp(1j * 0.9), g=g, eps=0.1)
        N = 7
    J = out["J"]
    rng = np.random.default_rng(1)
    sps = out["sps"]
    h = 1e-6
    for s in [sps[k] for k in rng.choice(len(sps), size=min(6, len(sps)), replace=False)]:
        theta = np.array(s["theta"])
        gV = rng.standard_normal()
        c = rng.standard_normal(N - 1)       # L = gV * V + c . theta
        dJ = O.xy_adjoint(N, J, theta, gV, c)
        assert np.allclose(dJ, dJ.T) and np.all(np.diag(dJ) == 0)
        for i, j in [(0, 1), (1, 3), (0, N - 1), (N - 2, N - 1)]:
            vals = []
            for sgn in (+1, -1):
                Jp = J.copy()
                Jp[i, j] += sgn * h
                Jp[j, i] += sgn * h
                tp = refine(theta, Jp)
                vals.append(gV * energy(tp, Jp) + c @ tp)
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(dJ[i, j] - fd) < 1e-6 * (1 + abs(fd)), (case, i, j, dJ[i, j], fd)


def test_adjoint_envelope_for_energy_alone():
    """With dL/dtheta = 0 the gradient is the envelope term 1 - cos(theta_i - theta_j)."""
    out = paper(7)
    J = out["J"]
    for s in out["sps"][:10]:
        th = np.append(s["theta"], 0.0)
        dJ = O.xy_adjoint(7, J, s["theta"], 1.0, None)
        expect = 1 - np.cos(th[:, None] - th[None, :])
        np.fill_diagonal(expect, 0.0)
        assert np.allclose(dJ, expect, atol=1e-15)
