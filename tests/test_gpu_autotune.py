"""The autotuner on the GPU: it picks launch shapes among its candidates, a solve with other
shapes gives the endpoints of the default shapes bit for bit (the knobs are scheduling
only); the step-control constants it picks pass its parity gate, and a solve with the
tuned options gives the default options' certified set; the second call is served from
the cache without launching anything."""
import numpy as np
import pytest

from gpu_common import nphc

pytestmark = pytest.mark.gpu


def test_tuned_shapes_change_no_result(tmp_path):
    N_ = nphc()
    from paper_1104_5497_gb300 import autotune as A
    from paper_1104_5497_gb300 import inputs as I
    inst = I.workload_n8()
    system = N_.System(inst.N, inst.sigma)
    opts = N_.options_default(gamma=inst.gamma)
    cache = str(tmp_path / "autotune.json")
    tuned, rep = A.tune(system, opts, sample=system.npaths, reps=1, cache=cache)
    assert not rep["cached"]
    assert rep["blocks_per_sm"] in A.FP32_CANDIDATES
    assert rep["list_blocks_per_sm"] in A.LIST_CANDIDATES + (0,)
    assert rep["threads_per_path"] in A.THREADS_PER_PATH
    assert set(rep["fp32_ms"]) == {str(c) for c in A.FP32_CANDIDATES}
    assert (rep["max_newton_fp32"], rep["eps_fp32"]) in A.STEP_CANDIDATES
    assert rep["step_gate"][f"{rep['threads_per_path']},{rep['max_newton_fp32']},{rep['eps_fp32']:g}"]
    # every other option is untouched
    assert (tuned.tol_sol, tuned.h_max, tuned.gamma_re) == (opts.tol_sol, opts.h_max, opts.gamma_re)
    # the tuned solve certifies the default solve's set (the gate covered every path)
    a, b = N_.solve(system, opts), N_.solve(system, tuned)
    ea, eb = a.endpoints(), b.endpoints()
    assert np.array_equal(ea["cls"], eb["cls"])
    c = np.isin(ea["cls"], [N_.END_REAL, N_.END_NONREAL])
    assert np.abs(ea["z"][c] - eb["z"][c]).max() <= 1e-10 * (1 + np.abs(ea["z"][c]).max())
    for shape in (dict(blocks_per_sm=4, list_blocks_per_sm=1), dict(blocks_per_sm=rep["blocks_per_sm"],
                                                                      list_blocks_per_sm=4)):
        a = N_.solve(system, opts).endpoints()
        b = N_.solve(system, A.apply(opts, shape)).endpoints()
        assert np.array_equal(a["status"], b["status"]) and np.array_equal(a["cls"], b["cls"])
        assert np.array_equal(a["z"], b["z"])   # bit for bit
    again, rep2 = A.tune(system, opts, cache=cache)
    assert rep2["cached"] and again.blocks_per_sm == tuned.blocks_per_sm
    assert A.tune(N_.System(6, 1.0), opts, cache=cache, measure=False)[1]["cached"] is False
