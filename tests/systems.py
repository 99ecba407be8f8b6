"""Generic quadratic systems with known solutions, as term lists (oracle.Terms), shared by
the oracle pins and the GPU tests of nphc_system_create_quadratic."""
import itertools

import numpy as np

import oracle as O


def x2_minus_5():
    # P(x) = x^2 - 5 as terms: 1 * x * x  +  (-5) * 1 * 1
    return O.Terms(1, [0, 0], [0, -1], [0, -1], [1.0, -5.0])


def product_system(n, seed):
    """P_i(z) = (w_i - a_i)(w_i - b_i) with w = A z: its 2^n roots are z = A^-1 w,
    w in prod_i {a_i, b_i}, all nonsingular when a_i != b_i and A is invertible."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 0.5 * np.eye(n)
    a = rng.standard_normal(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n) * (rng.random(n) < 0.5)
    eq, va, vb, co = [], [], [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                eq.append(i); va.append(j); vb.append(k); co.append(A[i, j] * A[i, k])
        for j in range(n):
            eq.append(i); va.append(j); vb.append(-1); co.append(-(a[i] + b[i]) * A[i, j])
        eq.append(i); va.append(-1); vb.append(-1); co.append(a[i] * b[i])
    roots = [np.linalg.solve(A, np.array(w)) for w in itertools.product(*zip(a, b))]
    return O.Terms(n, eq, va, vb, co), np.array(roots)


def random_quadratic(n, seed, density=1.0):
    """A random dense (or sparse) square quadratic system with complex coefficients:
    generically 2^n nonsingular isolated solutions (Bezout)."""
    rng = np.random.default_rng(seed)
    eq, va, vb, co = [], [], [], []
    for i in range(n):
        for j in range(-1, n):
            for k in range(j, n):
                if k < 0 or (j >= 0 and rng.random() > density):
                    continue
                eq.append(i); va.append(j); vb.append(k)
                co.append(complex(rng.standard_normal(), rng.standard_normal()))
        eq.append(i); va.append(-1); vb.append(-1)
        co.append(complex(rng.standard_normal(), rng.standard_normal()))
    return O.Terms(n, eq, va, vb, co)
