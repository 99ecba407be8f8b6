"""Each step of the method on its own through the C ABI, fed with the oracle's data:
classification of the oracle's real SPs, refinement/certification of the oracle's
endpoints, tracking of individual paths, deduplication of planted copies."""
import numpy as np
import pytest

import oracle as O
from gpu_common import nphc, oracle_xy, torus_dist
from paper_1104_5497_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def device_endpoints(N_, z, paths, cls=None, status=None):
    import torch
    z = np.asarray(z)
    ep = N_.DeviceEndpoints.empty(z.shape[1], paths)
    ep.tensors["z_re"].copy_(torch.from_numpy(np.ascontiguousarray(z.real.T)))
    ep.tensors["z_im"].copy_(torch.from_numpy(np.ascontiguousarray(z.imag.T)))
    if cls is not None:
        ep.tensors["cls"].copy_(torch.from_numpy(np.asarray(cls, np.int32)))
    if status is not None:
        ep.tensors["status"].copy_(torch.from_numpy(np.asarray(status, np.int32)))
    return ep


@pytest.mark.parametrize("N,sigma,seed", [(4, 1.5, 0), (5, 0.75, 10), (6, 1.5, 3), (7, 0.75, 12),
                                          (8, 1.5, 1)])
def test_classify_oracle_points(N, sigma, seed):
    import torch
    N_ = nphc()
    inst = I.ring(N, sigma, seed)
    ref = oracle_xy(N, sigma, inst.gamma.real, inst.gamma.imag)
    z = np.array([s["z"] for s in ref["sps"]])
    system = N_.System(N, sigma)
    ep = device_endpoints(N_, z, np.arange(len(z)), cls=np.full(len(z), N_.END_REAL))
    c = len(z)
    theta = torch.zeros(N - 1, c, dtype=torch.float64, device="cuda")
    index = torch.zeros(c, dtype=torch.int32, device="cuda")
    energy = torch.zeros(c, dtype=torch.float64, device="cuda")
    mineig = torch.zeros(c, dtype=torch.float64, device="cuda")
    logdet = torch.zeros(c, dtype=torch.float64, device="cuda")
    N_.classify(system, ep, theta, index, energy, mineig, logdet)
    torch.cuda.synchronize()
    th, ix, en, me = theta.cpu().numpy().T, index.cpu().numpy(), energy.cpu().numpy(), mineig.cpu().numpy()
    ld = logdet.cpu().numpy()
    for i, s in enumerate(ref["sps"]):
        assert torus_dist(th[i], s["theta"]) < 1e-12, i
        assert abs(en[i] - s["energy"]) < 1e-11, (i, en[i], s["energy"])
        assert abs(me[i] - s["min_abs_eig"]) < 1e-9 * (1 + s["min_abs_eig"]), (i, me[i], s["min_abs_eig"])
        assert abs(ld[i] - s["log_abs_det"]) < 1e-9 * (1 + abs(s["log_abs_det"])), (i, ld[i])
        assert ix[i] == s["index"], (i, ix[i], s["index"])


@pytest.mark.parametrize("N,sigma,seed", [(5, 0.75, 10), (7, 0.75, 12)])
def test_refine_certify_oracle_endpoints(N, sigma, seed):
    """Certification of the oracle's (already refined) endpoints gives the same class."""
    import torch
    N_ = nphc()
    inst = I.ring(N, sigma, seed)
    ref = oracle_xy(N, sigma, inst.gamma.real, inst.gamma.imag)
    system = N_.System(N, sigma)
    sel = np.nonzero(ref["status"] == O.REACHED)[0]
    ep = device_endpoints(N_, ref["z"][sel], sel, status=np.full(len(sel), N_.PATH_REACHED))
    opts = N_.options_default(gamma=inst.gamma)
    N_.refine_certify(system, opts, ep)
    torch.cuda.synchronize()
    cls = ep.tensors["cls"].cpu().numpy()
    assert np.array_equal(cls, ref["cls"][sel])
    zr = ep.tensors["z_re"].cpu().numpy().T + 1j * ep.tensors["z_im"].cpu().numpy().T
    cert = np.isin(cls, [N_.END_REAL, N_.END_NONREAL])
    d = np.linalg.norm(zr[cert] - ref["z"][sel][cert], axis=1)
    assert (d <= 1e-10 * (1 + np.linalg.norm(ref["z"][sel][cert], axis=1))).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_track_paths_match_oracle(prec):
    """Per path: every path the oracle tracks to a certified solution ends, on the GPU,
    at the same solution (the homotopy path from a given start point is unique)."""
    import torch
    N_ = nphc()
    N, sigma, seed = 6, 1.5, 3
    inst = I.ring(N, sigma, seed)
    ref = oracle_xy(N, sigma, inst.gamma.real, inst.gamma.imag)
    system = N_.System(N, sigma)
    P = 4 ** (N - 1)
    ep = N_.DeviceEndpoints.empty(2 * (N - 1), np.arange(P))
    ws = torch.zeros(system.workspace_size(P), dtype=torch.uint8, device="cuda")
    opts = N_.options_default(gamma=inst.gamma)
    N_.track(system, opts, N_.PREC_MIXED if prec == "mixed" else N_.PREC_FP64, ep, ws)
    N_.refine_certify(system, opts, ep)
    torch.cuda.synchronize()
    cls = ep.tensors["cls"].cpu().numpy()
    z = ep.tensors["z_re"].cpu().numpy().T + 1j * ep.tensors["z_im"].cpu().numpy().T
    cert_ref = np.isin(ref["cls"], [O.C_REAL, O.C_NONREAL])
    both = cert_ref & np.isin(cls, [N_.END_REAL, N_.END_NONREAL])
    same = np.linalg.norm(z[both] - ref["z"][both], axis=1) <= 1e-10 * (1 + np.linalg.norm(ref["z"][both], axis=1))
    assert both.sum() >= cert_ref.sum() - 2, (both.sum(), cert_ref.sum())
    assert same.mean() > 0.99


def test_dedup_flags_planted_copies():
    import torch
    N_ = nphc()
    N, sigma, seed = 5, 0.75, 10
    inst = I.ring(N, sigma, seed)
    ref = oracle_xy(N, sigma, inst.gamma.real, inst.gamma.imag)
    cert = np.nonzero(np.isin(ref["cls"], [O.C_REAL, O.C_NONREAL]))[0]
    # the certified endpoints, then copies of three of them under higher path indices
    sel = np.concatenate([cert, cert[[0, 5, 9]]])
    paths = np.concatenate([cert, 10 ** 6 + np.arange(3)])
    system = N_.System(N, sigma)
    ep = device_endpoints(N_, ref["z"][sel], paths, status=np.full(len(sel), N_.PATH_REACHED))
    opts = N_.options_default(gamma=inst.gamma)
    N_.refine_certify(system, opts, ep)
    ws = torch.zeros(system.workspace_size(len(sel)), dtype=torch.uint8, device="cuda")
    lst = torch.zeros(len(sel), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    N_.dedup(system, opts, ep, ws, lst, cnt)
    torch.cuda.synchronize()
    cls = ep.tensors["cls"].cpu().numpy()
    assert (cls[-3:] == N_.END_DUPLICATE).all()
    assert (cls[:-3] != N_.END_DUPLICATE).all()
    members = set(lst[:int(cnt.item())].cpu().numpy().tolist())
    assert members == {0, 5, 9, len(cert), len(cert) + 1, len(cert) + 2}


@pytest.mark.parametrize("N,sigma", [(8, 1.5), (9, 0.75)])
def test_refinement_scratch_matches_shared_memory(N, sigma):
    """The refinement keeps its Schur matrices in shared memory when called through
    nphc_refine_certify and in the result's global scratch inside nphc_solve_into: the
    arithmetic per endpoint is the same, so every endpoint the FP32 pass reached and both
    certify has bit-identical refined coordinates and the same class."""
    import torch
    N_ = nphc()
    inst = I.ring(N, sigma, 7)
    system = N_.System(N, sigma)
    opts = N_.options_default(gamma=inst.gamma, precision=N_.PREC_MIXED)
    full = N_.solve(system, opts).endpoints()
    P, n = system.npaths, system.n
    ep = N_.DeviceEndpoints.empty(n, np.arange(P))
    ws = torch.zeros(system.workspace_size(P), dtype=torch.uint8, device="cuda")
    N_.track(system, opts, N_.PREC_MIXED, ep, ws)
    reached = torch.nonzero(ep.tensors["status"] == N_.PATH_REACHED).flatten().to(torch.int32)
    count = torch.tensor([reached.numel()], dtype=torch.int32, device="cuda")
    N_.refine_certify(system, opts, ep, reached, count)
    torch.cuda.synchronize()
    cls = ep.tensors["cls"].cpu().numpy()
    z = (ep.tensors["z_re"] + 1j * ep.tensors["z_im"]).cpu().numpy().T
    idx = reached.cpu().numpy()
    certified = (N_.END_REAL, N_.END_NONREAL)
    both = [e for e in idx if cls[e] in certified and full["cls"][e] in certified]
    assert len(both) > 0.9 * sum(cls[e] in certified for e in idx), (len(both), len(idx))
    for e in both:
        assert cls[e] == full["cls"][e], e
        assert np.array_equal(z[e], full["z"][e]), (e, z[e], full["z"][e])


@pytest.mark.parametrize("N,sigma", [(7, 0.75), (9, 0.75)])
def test_solve_classification_matches_full_scan(N, sigma):
    """A solve classifies a compacted list of its real stationary points (32 to a warp);
    nphc_classify scans every entry.  The arithmetic per point is the same, so angles,
    indices, energies and log|det H| agree bit for bit, and every other entry of the scan
    has index -1."""
    import torch
    N_ = nphc()
    inst = I.ring(N, sigma, 11)
    system = N_.System(N, sigma)
    res = N_.solve(system, N_.options_default(gamma=inst.gamma))
    sps = res.stationary_points()
    full = res.endpoints()
    P = system.npaths
    ep = device_endpoints(N_, full["z"], np.arange(P), cls=full["cls"], status=full["status"])
    M = N - 1
    theta = torch.zeros(M, P, dtype=torch.float64, device="cuda")
    index = torch.zeros(P, dtype=torch.int32, device="cuda")
    energy = torch.zeros(P, dtype=torch.float64, device="cuda")
    logdet = torch.zeros(P, dtype=torch.float64, device="cuda")
    N_.classify(system, ep, theta, index, energy, None, logdet)
    torch.cuda.synchronize()
    th, ix, en, ld = theta.cpu().numpy().T, index.cpu().numpy(), energy.cpu().numpy(), logdet.cpu().numpy()
    real = full["cls"] == N_.END_REAL
    assert np.all(ix[~real] == -1)
    assert sorted(sps["path"].tolist()) == sorted(np.nonzero(real)[0].tolist())
    for i, e in enumerate(sps["path"]):
        assert np.array_equal(sps["theta"][i], th[e]), e
        assert sps["index"][i] == ix[e] and sps["energy"][i] == en[e] and sps["log_abs_det"][i] == ld[e], e
