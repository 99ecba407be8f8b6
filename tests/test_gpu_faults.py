"""Failures made on the host, on the GPU: a step budget of 1 ends every path of a plain
FP64 solve with NPHC_PATH_STEP_BUDGET (class NPHC_END_FAILED) instead of running on, and
the solve's counters say so; nothing hangs or faults."""
import numpy as np
import pytest

from gpu_common import nphc

pytestmark = pytest.mark.gpu


def test_step_budget_of_one_fails_every_path():
    N_ = nphc()
    system = N_.System(4, 1.5)
    res = N_.solve(system, N_.options_default(precision=N_.PREC_FP64, max_steps=1))
    ep, c = res.endpoints(), res.counts()
    assert np.all(ep["status"] == N_.PATH_STEP_BUDGET)
    assert np.all(ep["cls"] == N_.END_FAILED)
    assert (c["paths"], c["reached"], c["diverged"], c["failed"], c["real"]) == (64, 0, 0, 64, 0)
