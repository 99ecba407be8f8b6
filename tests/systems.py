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


# ---- systems with singular endpoints (Cauchy endgame pins), each with closed forms
def squares(n):
    """P_i = z_i^2: every path ends at z = 0.  Along the homotopy each coordinate solves
    (gamma (1-t) + t) z^2 = gamma (1-t), so z_i ~ +-sqrt(gamma (1-t)) near t = 1 and one
    turn around t = 1 swaps the two signs: cycle number 2."""
    return O.Terms(n, list(range(n)), list(range(n)), list(range(n)), [1.0] * n)


def double_root(a, b):
    """P_1 = (z_1 - a)^2, P_2 = z_2^2 - b: endpoints (a, +-sqrt(b)), each reached by two
    paths.  z_1 solves (gamma (1-t) + t) z^2 - 2 t a z + t a^2 - gamma (1-t) = 0, whose
    discriminant gamma (1-t) (gamma (1-t) + t (1 - a^2)) has a simple zero at t = 1 when
    a^2 != 1: cycle number 2 (z_2 is nonsingular, cycle 1)."""
    eq = [0, 0, 0, 1, 1]
    va = [0, 0, -1, 1, -1]
    vb = [0, -1, -1, 1, -1]
    co = [1.0, -2.0 * a, a * a, 1.0, -b]
    return O.Terms(2, eq, va, vb, co)


def chain4():
    """P_1 = z_1^2 - z_2, P_2 = z_2^2: every path ends at 0 with z_2 ~ (1-t)^(1/2) and
    z_1^2 ~ z_2, so z_1 ~ (1-t)^(1/4): cycle number 4."""
    return O.Terms(2, [0, 0, 1], [0, 1, 1], [0, -1, 1], [1.0, -1.0, 1.0])
