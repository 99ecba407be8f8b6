"""Stationary points as a differentiable function of the couplings (torch.autograd).

`stationary_points(J, gamma)` runs the whole method (nphc_solve) on the ring with
couplings J and returns the energies V* [K] and angles theta* [K, N-1] of its real
stationary points.  The backward pass is nphc_xy_adjoint: the envelope theorem for V*
and the implicit function theorem for theta* (one Hessian solve per point), so that any
loss built from V* and theta* can be differentiated with respect to J, and through J
with respect to sigma or the disorder when J is built from them with torch operations.
The set of stationary points is piecewise constant in J; the gradient is that of each
point followed continuously (the derivative of the method's outputs, not of the count).
"""
from __future__ import annotations

import numpy as np
import torch

from . import nphc


class _StationaryPoints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, J, gamma, opts):
        N = J.shape[0]
        Jh = J.detach().to("cpu", torch.float64).numpy()
        system = nphc.System(N, 1.0, Jh)
        res = nphc.solve(system, opts if opts is not None else nphc.options_default(gamma=gamma))
        sps = res.stationary_points()
        dev = J.device if J.is_cuda else torch.device("cuda")
        theta = torch.as_tensor(sps["theta"], dtype=torch.float64, device=dev)
        energy = torch.as_tensor(sps["energy"], dtype=torch.float64, device=dev)
        ctx.system = system
        ctx.save_for_backward(theta)
        ctx.jdev, ctx.jdtype = J.device, J.dtype
        return energy.to(J.device), theta.to(J.device)

    @staticmethod
    def backward(ctx, g_energy, g_theta):
        (theta,) = ctx.saved_tensors
        dev = theta.device
        ge = None if g_energy is None else g_energy.to(dev, torch.float64)
        gt = None if g_theta is None else g_theta.to(dev, torch.float64)
        dJ = nphc.xy_adjoint(ctx.system, theta, ge, gt)
        # nphc_xy_adjoint gives dL/dJ_ij of the one parameter J_ij = J_ji on both entries;
        # as a function of the matrix entries (a symmetric perturbation moves both) each
        # entry carries half of it
        return (0.5 * dJ).to(ctx.jdev, ctx.jdtype), None, None


def stationary_points(J: torch.Tensor, gamma: complex = np.exp(0.5j), opts=None):
    """(energy [K], theta [K, N-1]) of the real stationary points of the ring with
    couplings J (symmetric N x N, zero diagonal), differentiable with respect to J."""
    return _StationaryPoints.apply(J, gamma, opts)


def ring_couplings(N: int, sigma: torch.Tensor) -> torch.Tensor:
    """J_ij = d_ij^-sigma with d_ij = min(|i-j|, N-|i-j|), as a torch function of sigma."""
    i = torch.arange(N, dtype=torch.float64, device=sigma.device)
    d = (i[:, None] - i[None, :]).abs()
    d = torch.minimum(d, N - d)
    off = d > 0
    J = torch.zeros(N, N, dtype=torch.float64, device=sigma.device)
    J[off] = d[off] ** (-sigma)
    return J
