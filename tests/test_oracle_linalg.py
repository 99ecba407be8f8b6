"""Pins for the oracle's textbook linear algebra against numpy/LAPACK."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 14, 18, 22])
def test_lu_solve_matches_lapack(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x = O.lu_solve(A, b)
        ref = np.linalg.solve(A, b)
        assert np.abs(x - ref).max() <= 1e-10 * (1 + np.abs(ref).max())


def test_lu_needs_pivoting():
    # a zero leading entry forces a row interchange
    A = np.array([[0, 1, 2], [3, 0, 1], [1, 1, 0]], dtype=complex)
    b = np.array([1, 2, 3], dtype=complex)
    assert np.allclose(O.lu_solve(A, b), np.linalg.solve(A, b), atol=1e-14)


def test_lu_singular_is_reported():
    A = np.array([[1, 2], [2, 4]], dtype=complex)
    with pytest.raises(np.linalg.LinAlgError):
        O.lu_solve(A, np.ones(2))


@pytest.mark.parametrize("n", [1, 2, 4, 9, 11])
def test_jacobi_eigenvalues_match_lapack(n):
    rng = np.random.default_rng(100 + n)
    M = rng.standard_normal((n, n))
    A = M + M.T
    assert np.allclose(O.sym_eig(A), np.linalg.eigvalsh(A), atol=1e-12)
