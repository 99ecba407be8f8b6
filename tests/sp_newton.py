"""Newton's method on grad V for one stationary point of the XY ring, written from V's
definition (independent of the oracle and of the CUDA path): follows a stationary point
under perturbed couplings for finite-difference checks of gradients."""
import numpy as np


def grad_hess(theta, J):
    """grad and Hessian of V = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)) in the free
    angles (theta_N = 0 appended)."""
    N = len(J)
    th = np.append(theta, 0.0)
    D = th[:, None] - th[None, :]
    G = (J * np.sin(D)).sum(axis=1)[:-1]
    C = J * np.cos(D)
    H = -C[:-1, :-1].copy()
    np.fill_diagonal(H, C.sum(axis=1)[:-1] - np.diag(C)[:-1])
    return G, H


def energy(theta, J):
    th = np.append(theta, 0.0)
    D = th[:, None] - th[None, :]
    return 0.5 * (J * (1 - np.cos(D))).sum()


def refine(theta, J, iters=30):
    for _ in range(iters):
        G, H = grad_hess(theta, J)
        theta = theta - np.linalg.solve(H, G)
    assert np.abs(grad_hess(theta, J)[0]).max() < 1e-12
    return theta
