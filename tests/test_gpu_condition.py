"""The condition-estimate hand-off of the mixed-precision pipeline: a converged FP32 step
whose Schur system's condition estimate (max |U_kk| / min |U_kk| of its pivoted LU factor)
exceeds kappa_fp32 is not taken, and FP64 continues the path from its last accepted
point.  Those paths end in FP64, and the certified set is the oracle's whatever the
threshold."""
import numpy as np
import pytest

from gpu_common import assert_same_point_sets, certified_set, nphc, oracle_xy
import oracle as O
from paper_1104_5497_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_low_threshold_hands_paths_to_fp64_in_the_step_calls():
    """nphc_track in MIXED precision with a low kappa_fp32 stops paths with
    NPHC_PATH_HANDOFF_COND; an FP64 call with resume = 1 takes every one of them to an
    FP64 end (reached, diverged, or the minimum step at the ring's singular solution
    sets), none left running or handed off."""
    import torch
    N_ = nphc()
    inst = I.workload_n8()
    M = inst.N - 1
    P = 4 ** M
    system = N_.System(inst.N, inst.sigma)
    ep = N_.DeviceEndpoints.empty(2 * M, np.arange(P))
    ws = torch.zeros(system.workspace_size(P), dtype=torch.uint8, device="cuda")
    opts = N_.options_default(gamma=inst.gamma, kappa_fp32=1e3)
    N_.track(system, opts, N_.PREC_MIXED, ep, ws)
    torch.cuda.synchronize()
    st = ep.tensors["status"]
    cond = torch.nonzero(st == N_.PATH_HANDOFF_COND).flatten().to(torch.int32)
    assert cond.numel() > 0
    n = torch.tensor([cond.numel()], dtype=torch.int32, device="cuda")
    N_.track(system, opts, N_.PREC_FP64, ep, ws, cond, n, resume=True)
    torch.cuda.synchronize()
    end = ep.tensors["status"][cond.long()].cpu().numpy()
    assert not np.isin(end, [N_.PATH_RUNNING, N_.PATH_HANDOFF, N_.PATH_HANDOFF_COND]).any()
    assert (end == N_.PATH_REACHED).sum() > 0 and (end == N_.PATH_DIVERGED).sum() > 0
    # with the test off no path stops for that reason
    N_.track(system, N_.options_default(gamma=inst.gamma, kappa_fp32=0.0), N_.PREC_MIXED, ep, ws)
    torch.cuda.synchronize()
    assert int((ep.tensors["status"] == N_.PATH_HANDOFF_COND).sum()) == 0


@pytest.mark.parametrize("kappa", [1e4, 3e5, 1e6])
def test_certified_set_unchanged_by_the_threshold(kappa):
    """The N = 8 workload (16,384 paths) in mixed precision with kappa_fp32 = 1e4, the
    default 3e5 and 1e6: the condition test hands paths to FP64 (counted), and the
    certified real and non-real sets are the oracle's."""
    N_ = nphc()
    inst = I.workload_n8()
    system = N_.System(inst.N, inst.sigma)
    res = N_.solve(system, N_.options_default(gamma=inst.gamma, kappa_fp32=kappa))
    c = res.counts()
    if kappa == 1e4:
        assert c["handoff_cond"] > 0
    assert c["handoff_cond"] <= c["handoff"]
    ep = res.endpoints()
    ref = oracle_xy(inst.N, float(inst.sigma), float(np.real(inst.gamma)), float(np.imag(inst.gamma)))
    for cl_gpu, cl_or in ((N_.END_REAL, O.C_REAL), (N_.END_NONREAL, O.C_NONREAL)):
        assert_same_point_sets(certified_set(ep["z"], ep["cls"], [cl_gpu]),
                               certified_set(ref["z"], ref["cls"], [cl_or]))
