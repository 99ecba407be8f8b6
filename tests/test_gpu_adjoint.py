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


def test_n12_ground_state_and_lowest_saddle_gradients():
    """The N = 12 ring at sigma = 1 (22 unknowns, 4,194,304 paths): the ground state and
    the lowest index-1 saddle.  dE/dsigma (through ring_couplings) and dE/dJ_ij for every
    pair (the adjoint) against central differences that follow each point by Newton's
    method under the perturbed couplings, within 1e-6 relative (of the gradient's largest
    entry); the ground state's gradient is zero (V = 0 at theta = 0 for every coupling)."""
    import torch
    from paper_1104_5497_gb300.autograd import ring_couplings, stationary_points
    from sp_newton import grad_hess
    nphc()
    inst = I.workload_n12()
    N = inst.N
    sigma = torch.tensor(inst.sigma, dtype=torch.float64, device="cuda", requires_grad=True)
    J = ring_couplings(N, sigma)
    V, theta = stationary_points(J, inst.gamma)
    assert len(V) >= 9297                     # a random-start search's lower bound
    Vh, th = V.detach().cpu().numpy(), theta.detach().cpu().numpy()
    J0 = O.couplings(N, inst.sigma)
    order = np.argsort(Vh)
    k0 = int(order[0])
    assert abs(Vh[k0]) < 1e-12 and np.abs(np.angle(np.exp(1j * th[k0]))).max() < 1e-12
    k1 = None
    for k in order[1:]:
        ev = np.linalg.eigvalsh(grad_hess(th[k], J0)[1])
        if (ev < 0).sum() == 1:
            k1 = int(k)
            break
    assert k1 is not None
    iu = np.triu_indices(N, 1)
    for k in (k0, k1):
        gs, gJ = torch.autograd.grad(V[k], [sigma, J], retain_graph=True)
        gs = float(gs)
        gJ = gJ.cpu().numpy()[iu]
        h = 1e-6

        def e_at(Jp):
            return energy(refine(th[k].copy(), Jp), Jp)
        fd_s = (e_at(O.couplings(N, inst.sigma + h)) - e_at(O.couplings(N, inst.sigma - h))) / (2 * h)
        fd_J = np.zeros(len(iu[0]))
        for q, (i, j) in enumerate(zip(*iu)):
            Jp, Jm = J0.copy(), J0.copy()
            Jp[i, j] = Jp[j, i] = J0[i, j] + h
            Jm[i, j] = Jm[j, i] = J0[i, j] - h
            fd_J[q] = (e_at(Jp) - e_at(Jm)) / (2 * h)
        if k == k0:
            assert abs(gs) <= 1e-15 and np.abs(gJ).max() <= 1e-15
            assert abs(fd_s) < 1e-9 and np.abs(fd_J).max() < 1e-9
        else:
            assert Vh[k] > 0
            assert abs(gs - fd_s) <= 1e-6 * abs(fd_s), (gs, fd_s)
            assert np.abs(gJ - fd_J).max() <= 1e-6 * np.abs(fd_J).max()
