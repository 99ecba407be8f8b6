"""The index histograms of the real stationary points, pinned by Morse theory: with
theta_N pinned, V is a function on the torus T^(N-1), and when every critical point is
nondegenerate (true for the rings below; not for uniform rings with N = 0 mod 4, whose
critical sets include circles) the counts c_k of critical points of index k satisfy
  sum_k (-1)^k c_k = chi(T^(N-1)) = 0,
  c_k >= b_k = C(N-1, k)                                  (weak Morse inequalities),
  sum_{k<=j} (-1)^(j-k) (c_k - b_k) >= 0 for every j     (strong Morse inequalities).
A lost stationary point, or one given the wrong index, breaks the first relation unless
another error compensates it exactly.  The paper prints none of the histograms."""
from math import comb

import numpy as np
import pytest

import oracle as O
from oracle_cases import paper, xy


def index_hist(out, N):
    h = np.zeros(N, int)
    for s in out["sps"]:
        h[s["index"]] += 1
    return h


def check_morse(h, N):
    m = N - 1
    b = [comb(m, k) for k in range(m + 1)]
    assert sum((-1) ** k * int(h[k]) for k in range(m + 1)) == 0, h
    assert all(h[k] >= b[k] for k in range(m + 1)), h
    for j in range(m + 1):
        assert sum((-1) ** (j - k) * (int(h[k]) - b[k]) for k in range(j + 1)) >= 0, (j, h)


@pytest.mark.parametrize("N", [3, 5, 7, 9])
def test_paper_rings(N):
    check_morse(index_hist(paper(N), N), N)


@pytest.mark.parametrize("N,sigma,seed", [(5, 1.0, 1), (6, 1.5, 3), (7, 2.0, 2)])
def test_power_law_rings(N, sigma, seed):
    check_morse(index_hist(xy(N, sigma, seed), N), N)


def test_disordered_ring_n8():
    """Disorder breaks the symmetry that makes the uniform N = 8 ring degenerate."""
    N = 8
    rng = np.random.default_rng(4)
    g = rng.standard_normal((N, N))
    g = np.triu(g, 1) + np.triu(g, 1).T
    out = O.solve_xy(N, 1.2, np.exp(0.9j), g=g, eps=0.1)
    assert (out["cls"] == O.C_SINGULAR).sum() == 0
    check_morse(index_hist(out, N), N)


def test_a_lost_saddle_breaks_the_relation():
    h = index_hist(paper(7), 7)
    h[3] -= 1
    with pytest.raises(AssertionError):
        check_morse(h, 7)
