"""Adjoint gradients on the GPU (nphc_xy_adjoint and the torch.autograd wrapper) against
the oracle's adjoint and against finite differences that follow each stationary point
under perturbed couplings."""
import numpy as np
import pytest

import oracle as O
from gpu_common import nphc
from oracle_cases import paper
from paper_1104_5497_gb300 import inputs as I
from sp_newton import energy, refine

pytestmark = pytest.mark.gpu


def test_adjoint_kernel_matches_oracle():
    import torch
    N_ = nphc()
    N = 7
    out = paper(N)
    inst = I.paper_ring(N)
    system = N_.System(N, inst.sigma)
    res = N_.solve(system, N_.options_default(gamma=inst.gamma))
    sps = res.stationary_points()
    K = len(sps["theta"])
    assert K == 168
    rng = np.random.default_rng(2)
    ge, gt = rng.standard_normal(K), rng.standard_normal((K, N - 1))
    th = torch.as_tensor(sps["theta"], device="cuda")
    dJ = N_.xy_adjoint(system, th, torch.as_tensor(ge, device="cuda"),
                       torch.as_tensor(gt, device="cuda")).cpu().numpy()
    ref = sum(O.xy_adjoint(N, out["J"], sps["theta"][k], ge[k], gt[k]) for k in range(K))
    assert np.abs(dJ - ref).max() <= 1e-9 * (1 + np.abs(ref).max())
    # energy-only cotangents: the envelope term alone
    dJe = N_.xy_adjoint(system, th, torch.ones(K, dtype=torch.float64, device="cuda")).cpu().numpy()
    refe = sum(O.xy_adjoint(N, out["J"], sps["theta"][k], 1.0) for k in range(K))
    assert np.abs(dJe - refe).max() <= 1e-12 * (1 + np.abs(refe).max())


def test_autograd_sigma_gradient_matches_finite_differences():
    """L = sum_k V_k + c . theta_k over the real SPs of the N = 8 ring: dL/dsigma through
    J(sigma) = d^-sigma and the adjoint equals the central difference in sigma with every
    SP Newton-refined under the perturbed couplings."""
    import torch
    from paper_1104_5497_gb300.autograd import ring_couplings, stationary_points
    nphc()
    inst = I.workload_n8()
    N = inst.N
    sigma = torch.tensor(inst.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    J = ring_couplings(N, sigma)
    V, theta = stationary_points(J, inst.gamma)
    rng = np.random.default_rng(5)
    c = torch.as_tensor(rng.standard_normal(N - 1), device="cuda")
    L = V.sum() + (theta * c).sum()
    L.backward()
    grad = float(sigma.grad)
    th0 = theta.detach().cpu().numpy()
    cc = c.cpu().numpy()
    h = 1e-6
    vals = []
    for sgn in (+1, -1):
        Jp = ring_couplings(N, torch.tensor(inst.sigma + sgn * h, dtype=torch.float64)).numpy()
        tot = 0.0
        for t in th0:
            tp = refine(t, Jp)
            tot += energy(tp, Jp) + cc @ tp
        vals.append(tot)
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(grad - fd) < 1e-6 * (1 + abs(fd)), (grad, fd)
