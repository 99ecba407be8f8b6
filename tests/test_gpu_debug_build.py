"""The debug build (NPHC_DEBUG, `build.build_debug()`): every kernel checks its work-list,
list-append, dedup-link and batch-item indices, records the first failure for
nphc_debug_check and skips the access.  Small solves through it record no failure and
give the release build's results; a work list with an entry beyond the endpoint set is
caught (code 1) while the valid entries are tracked.  The debug library runs in a child
process (one library per process)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_common import nphc
from paper_1104_5497_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[2])
import paper_1104_5497_gb300.nphc as N_
from paper_1104_5497_gb300 import inputs as I
N_.use_library(sys.argv[1])
out = {"codes": []}
def note():
    out["codes"].append(N_.debug_check())
def summary(c):
    return {k: c[k] for k in ("paths", "real", "nonreal", "singular", "duplicate", "failed", "handoff")}
for N, sigma, seed in ((4, 1.5, 0), (5, 0.75, 10)):
    inst = I.ring(N, sigma, seed)
    for prec in (N_.PREC_MIXED, N_.PREC_FP64):
        r = N_.solve(N_.System(N, sigma), N_.options_default(gamma=inst.gamma, precision=prec))
        out[f"ring{N}_{prec}"] = summary(r.counts())
        note()
insts = I.disordered_batch(4, seed=3)
B = N_.Batch([N_.System(b.N, b.sigma, N_.xy_couplings(b.N, b.sigma, b.g, b.eps)) for b in insts])
B.solve([N_.options_default(gamma=b.gamma) for b in insts])
out["batch"] = [summary(B.result(i).counts()) for i in range(len(insts))]
note()
# a planted entry beyond the endpoint set: the arrays are padded far past it
N = 4; M = N - 1; n = 2 * M; count = 16
pad = N_.DeviceEndpoints.empty(n, np.arange(count + 64))
ep = N_.DeviceEndpoints(count, n, {k: v for k, v in pad.tensors.items()})
system = N_.System(N, 1.5)
ws = torch.zeros(system.workspace_size(count + 64), dtype=torch.uint8, device="cuda")
lst = torch.tensor([0, 1, count + 5], dtype=torch.int32, device="cuda")
cnt = torch.tensor([3], dtype=torch.int32, device="cuda")
N_.track(system, N_.options_default(), N_.PREC_FP64, ep, ws, lst, cnt)
torch.cuda.synchronize()
out["planted_code"] = N_.debug_check()
out["planted_status"] = ep.tensors["status"][:2].cpu().tolist()
print(json.dumps(out))
"""


def test_debug_build_checks_indices():
    N_ = nphc()
    from paper_1104_5497_gb300 import build
    dbg = build.build_debug()
    r = subprocess.run([sys.executable, "-c", CHILD, dbg, ROOT], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert got["codes"] and all(c == 0 for c in got["codes"]), got["codes"]
    assert got["planted_code"] == 1
    assert all(s in (N_.PATH_REACHED, N_.PATH_DIVERGED) for s in got["planted_status"])
    assert N_.debug_check() == -1   # this process runs the release build
    # the release build's results
    for N, sigma, seed in ((4, 1.5, 0), (5, 0.75, 10)):
        inst = I.ring(N, sigma, seed)
        for prec in (N_.PREC_MIXED, N_.PREC_FP64):
            c = N_.solve(N_.System(N, sigma), N_.options_default(gamma=inst.gamma, precision=prec)).counts()
            assert got[f"ring{N}_{prec}"] == {k: c[k] for k in got[f"ring{N}_{prec}"]}
