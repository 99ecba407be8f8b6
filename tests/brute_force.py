"""Brute-force real stationary points of the power-law XY ring, independent of homotopy.

Test helper.  Newton's method on grad V in the angles themselves (no polynomial
system, no homotopy, no complex arithmetic), started from every point of a regular
angle grid plus uniform random starts, all at once with numpy.  It works from the
potential as the paper writes it (section "A First Application"):

    V(theta) = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)),  theta_N = 0,
    dV/dtheta_k = sum_j J_kj sin(theta_k - theta_j),
    d2V/dtheta_k^2 = sum_{j != k} J_kj cos(theta_k - theta_j),
    d2V/dtheta_k dtheta_l = -J_kl cos(theta_k - theta_l).

It returns the nonsingular real stationary points it finds (each once), with their
Hessian index; for small N a fine grid reaches every basin, so the set is complete.
The couplings are built here too, straight from d_ij = min(|i-j|, N-|i-j|).
"""
from __future__ import annotations

import numpy as np


def ring_couplings(N: int, sigma: float, g: np.ndarray | None = None, eps: float = 0.1) -> np.ndarray:
    i = np.arange(N)
    d = np.abs(i[:, None] - i[None, :])
    d = np.minimum(d, N - d).astype(float)
    with np.errstate(divide="ignore"):
        J = np.where(d > 0, d ** (-float(sigma)), 0.0)
    if g is not None:
        J = J * (1.0 + eps * g)
        np.fill_diagonal(J, 0.0)
    return J


def grad_hess(theta: np.ndarray, J: np.ndarray):
    """theta: (S, m) free angles.  Returns grad (S, m) and Hessian (S, m, m)."""
    S, m = theta.shape
    th = np.concatenate([theta, np.zeros((S, 1))], axis=1)          # theta_N = 0
    D = th[:, :, None] - th[:, None, :]
    g = (J[None] * np.sin(D)).sum(axis=2)[:, :m]
    C = J[None] * np.cos(D)
    H = -C[:, :m, :m].copy()
    diag = C.sum(axis=2)[:, :m]                                        # J_kk = 0
    idx = np.arange(m)
    H[:, idx, idx] = diag
    return g, H


def energy(theta: np.ndarray, J: np.ndarray) -> np.ndarray:
    S = theta.shape[0]
    th = np.concatenate([theta, np.zeros((S, 1))], axis=1)
    D = th[:, :, None] - th[:, None, :]
    return 0.5 * (J[None] * (1.0 - np.cos(D))).sum(axis=(1, 2))


def real_stationary_points(N: int, J: np.ndarray, grid: int = 16, n_random: int = 0,
                           seed: int = 0, iters: int = 60, sing_tol: float = 1e-7):
    """Nonsingular real SPs found from a grid^(N-1) angle grid (+ random starts).

    Returns (theta (K, m) in (-pi, pi], index (K,), energy (K,), n_singular_hits)."""
    m = N - 1
    ax = -np.pi + (np.arange(grid) + 0.5) * (2 * np.pi / grid)
    starts = np.stack(np.meshgrid(*([ax] * m), indexing="ij"), axis=-1).reshape(-1, m)
    if n_random:
        rng = np.random.default_rng(seed)
        starts = np.concatenate([starts, rng.uniform(-np.pi, np.pi, (n_random, m))])
    th = starts.copy()
    for _ in range(iters):
        g, H = grad_hess(th, J)
        ok = np.abs(np.linalg.det(H)) > 1e-300
        step = np.zeros_like(th)
        step[ok] = np.linalg.solve(H[ok], g[ok][..., None])[..., 0]
        th = th - np.clip(step, -1.0, 1.0)   # damped far from a root, plain Newton near one
    g, H = grad_hess(th, J)
    conv = np.linalg.norm(g, axis=1) < 1e-11
    th = th[conv]
    H = H[conv]
    ev = np.linalg.eigvalsh(H)
    scale = np.abs(J).sum()
    nonsing = np.abs(ev).min(axis=1) > sing_tol * scale
    n_sing = int((~nonsing).sum())
    th = np.angle(np.exp(1j * th[nonsing]))
    th[np.abs(th + np.pi) < 1e-9] = np.pi
    ev = ev[nonsing]
    # one representative per distinct point on the torus
    keep = []
    for i in range(len(th)):
        if not any(np.abs(np.angle(np.exp(1j * (th[i] - th[k])))).max() < 1e-7 for k in keep):
            keep.append(i)
    th = th[keep]
    index = (ev[keep] < 0).sum(axis=1)
    return th, index, energy(th, J), n_sing
