"""Stationary points as a differentiable function of the couplings (torch.autograd).

`stationary_points(J, gamma)` runs the whole method (nphc_solve) on the ring with
couplings J and returns the energies V* [K] and angles theta* [K, N-1] of its real
stationary points.  The backward pass is nphc_xy_adjoint: the envelope theorem for V*
and the implicit function theorem for theta* (one Hessian solve per point).  The
couplings are the N(N-1)/2 entries above the diagonal (J_ij = J_ji is one parameter), so
the gradient with respect to the matrix reaches its upper triangle.  `ring_couplings`
builds J_ij = d_ij^-sigma (1 + eps g_ij) with nphc_xy_couplings, and its backward pass is
nphc_xy_couplings_vjp, so dL/dsigma of any loss on the stationary points follows.  Every
number is computed by the library; this module only moves arrays between torch and the
C ABI.  The set of stationary points is piecewise constant in J; the gradient is that of
each point followed continuously (the derivative of the method's outputs, not of the
count).
"""
from __future__ import annotations

import numpy as np
import torch

from . import nphc


def _upper(N: int):
    return np.triu_indices(N, 1)


class _StationaryPoints(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, N, gamma, opts):
        iu = _upper(N)
        Jh = np.zeros((N, N))
        ph = p.detach().to("cpu", torch.float64).numpy()
        Jh[iu] = ph                 # the system is built on the host (a small matrix)
        Jh[iu[1], iu[0]] = ph
        system = nphc.System(N, 1.0, Jh)
        res = nphc.solve(system, opts if opts is not None else nphc.options_default(gamma=gamma))
        sps = res.stationary_points()
        dev = p.device if p.is_cuda else torch.device("cuda")
        theta = torch.as_tensor(sps["theta"], dtype=torch.float64, device=dev)
        energy = torch.as_tensor(sps["energy"], dtype=torch.float64, device=dev)
        ctx.system = system
        ctx.N = N
        ctx.save_for_backward(theta)
        ctx.pdev, ctx.pdtype = p.device, p.dtype
        return energy.to(p.device), theta.to(p.device)

    @staticmethod
    def backward(ctx, g_energy, g_theta):
        (theta,) = ctx.saved_tensors
        dev = theta.device
        ge = None if g_energy is None else g_energy.to(dev, torch.float64)
        gt = None if g_theta is None else g_theta.to(dev, torch.float64)
        dJ = nphc.xy_adjoint(ctx.system, theta, ge, gt)   # dL/dJ_ij of each pair parameter
        iu = _upper(ctx.N)
        rows = torch.as_tensor(iu[0], device=dev)
        cols = torch.as_tensor(iu[1], device=dev)
        return dJ[rows, cols].to(ctx.pdev, ctx.pdtype), None, None, None


def stationary_points(J: torch.Tensor, gamma: complex = np.exp(0.5j), opts=None):
    """(energy [K], theta [K, N-1]) of the real stationary points of the ring with
    couplings J (symmetric N x N, zero diagonal: its upper triangle is read),
    differentiable with respect to J."""
    N = J.shape[0]
    iu = _upper(N)
    p = J[torch.as_tensor(iu[0], device=J.device), torch.as_tensor(iu[1], device=J.device)]
    return _StationaryPoints.apply(p, N, gamma, opts)


class _RingCouplings(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma, N, g, eps):
        s = float(sigma.detach().cpu())
        J = nphc.xy_couplings(N, s, g, eps)
        ctx.args = (N, s, g, eps)
        ctx.sdev, ctx.sdtype = sigma.device, sigma.dtype
        return torch.as_tensor(J, dtype=torch.float64, device=sigma.device)

    @staticmethod
    def backward(ctx, grad_J):
        N, s, g, eps = ctx.args
        ds = nphc.xy_couplings_vjp(N, s, grad_J.detach().to("cpu", torch.float64).numpy(), g, eps)
        return torch.tensor(ds, dtype=ctx.sdtype, device=ctx.sdev), None, None, None


def ring_couplings(N: int, sigma: torch.Tensor, g: np.ndarray | None = None,
                   eps: float = 0.1) -> torch.Tensor:
    """J_ij = d_ij^-sigma (1 + eps g_ij) (nphc_xy_couplings), d_ij = min(|i-j|, N-|i-j|), as a
    torch function of the scalar tensor sigma."""
    return _RingCouplings.apply(sigma, N, g, eps)
