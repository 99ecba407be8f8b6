"""Batches of independent systems (nphc_batch_*): the 64-instance disordered workload
(N = 6..9, one gamma per instance) solved together -- one FP32 launch per ring size over a
global (instance, path) queue, or every instance on its own stream -- eagerly and through
one captured CUDA graph, gives every instance the same results as solving it alone;
every instance with N <= 7 is checked against the oracle point by point."""
import numpy as np
import pytest

import oracle as O
from gpu_common import assert_same_point_sets, certified_set, nphc
from paper_1104_5497_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def instance_system(N_, inst):
    J = N_.xy_couplings(inst.N, inst.sigma, inst.g, inst.eps)
    return N_.System(inst.N, inst.sigma, J)


def certified(res, N_):
    ep = res.endpoints()
    c = np.isin(ep["cls"], [N_.END_REAL, N_.END_NONREAL])
    z = ep["z"][c]
    return z[np.lexsort(np.round(np.concatenate([z.real, z.imag], axis=1).T, 8))]


@pytest.mark.parametrize("per_instance", [False, True])
def test_batch64_matches_single_solves_and_graph_replays(per_instance):
    N_ = nphc()
    insts = I.workload_batch64()
    assert len(insts) == 64
    systems = [instance_system(N_, inst) for inst in insts]
    opts = [N_.options_default(gamma=inst.gamma) for inst in insts]
    batch = N_.Batch(systems)
    for mode in ("eager", "capture", "replay"):
        batch.solve(opts, graph=(mode != "eager"), per_instance=per_instance)
        for i in (0, 5, 17, 33, 40, 63):
            single = N_.solve(systems[i], opts[i])
            a, b = batch.result(i).counts(), single.counts()
            for k in ("paths", "real", "nonreal", "duplicate", "index_hist"):
                assert a[k] == b[k], (mode, i, k, a[k], b[k])
            za, zb = certified(batch.result(i), N_), certified(single, N_)
            assert za.shape == zb.shape
            assert np.abs(za - zb).max() <= 1e-9 * (1 + np.abs(zb).max())


def test_batch_instances_match_the_oracle():
    """Every instance of the 64-ring workload with N <= 7 (27 rings, grouped launches
    and a captured graph): the certified real and non-real sets equal the oracle's, one to
    one within 1e-10 relative."""
    N_ = nphc()
    insts = [inst for inst in I.workload_batch64() if inst.N <= 7]
    assert len(insts) >= 20
    systems = [instance_system(N_, inst) for inst in insts]
    opts = [N_.options_default(gamma=inst.gamma) for inst in insts]
    batch = N_.Batch(systems)
    batch.solve(opts)
    batch.solve(opts, graph=True)
    for i, inst in enumerate(insts):
        ref = O.solve_xy(inst.N, inst.sigma, inst.gamma, g=inst.g, eps=inst.eps)
        ep = batch.result(i).endpoints()
        for cl_gpu, cl_or in ((N_.END_REAL, O.C_REAL), (N_.END_NONREAL, O.C_NONREAL)):
            assert_same_point_sets(certified_set(ep["z"], ep["cls"], [cl_gpu]),
                                   certified_set(ref["z"], ref["cls"], [cl_or]))


def test_batch_with_endgame_matches_single_solves():
    """opts.endgame inside a batch (eager, captured, replayed): every instance gets the
    endgame outcomes of its single solve (rings with N = 0 mod 4 have singular endpoints;
    the other instances have none)."""
    N_ = nphc()
    rings = [(8, 1.0, np.exp(0.5j)), (4, 1.5, np.exp(1.1j)), (8, 1.5, np.exp(2.3j)), (6, 1.0, np.exp(0.5j))]
    systems = [N_.System(N, s) for N, s, _ in rings]
    opts = [N_.options_default(gamma=g, endgame=1) for _, _, g in rings]
    batch = N_.Batch(systems)
    singles = [N_.solve(s, o) for s, o in zip(systems, opts)]
    for mode in ("eager", "capture", "replay"):
        batch.solve(opts, graph=(mode != "eager"))
        for i, single in enumerate(singles):
            a, b = batch.result(i).counts(), single.counts()
            for k in ("eg_run", "eg_converged", "eg_multiple", "eg_at_infinity", "singular", "failed"):
                assert a[k] == b[k], (mode, i, k, a[k], b[k])
            ea, eb = batch.result(i).endgame(), single.endgame()
            assert np.array_equal(ea["status"], eb["status"]) and np.array_equal(ea["cycle"], eb["cycle"])
            conv = eb["status"] == N_.EG_CONVERGED
            za, zb = batch.result(i).endpoints()["z"][conv], single.endpoints()["z"][conv]
            if conv.any():
                assert np.abs(za - zb).max() <= 1e-9 * (1 + np.abs(zb).max())
    assert singles[0].counts()["eg_converged"] > 0
