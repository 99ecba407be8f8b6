"""nphc_dedup_noalloc (deduplication with the library's fixed scratch array instead of a
caller workspace) against nphc_dedup, through the C ABI.

The file name sorts last so that pytest collects it after the other tests: the fixed
array then already holds an earlier call's contents when a test here runs, and it must
give the same answer as when it runs alone in a fresh process."""
import numpy as np
import pytest

from gpu_common import nphc
from paper_1104_5497_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _select(N_, ep, idx, paths):
    """A new endpoint set: the entries idx of ep under new path indices."""
    import torch
    idx = torch.as_tensor(idx, dtype=torch.int64, device="cuda")
    out = N_.DeviceEndpoints.empty(ep.n, paths)
    for k, v in ep.tensors.items():
        if k == "path":
            continue
        out.tensors[k].copy_(v.index_select(v.dim() - 1, idx))
    return out


def _clone(N_, ep):
    out = N_.DeviceEndpoints.empty(ep.n, ep.tensors["path"].clone())
    for k, v in ep.tensors.items():
        out.tensors[k].copy_(v)
    return out


def _run(N_, system, opts, ep, noalloc):
    """Dedup a fresh copy of ep; returns (cls, set of dup_list entries, dup_count)."""
    import torch
    e = _clone(N_, ep)
    lst = torch.full((e.count,), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    if noalloc:
        N_.dedup_noalloc(system, opts, e, lst, cnt)
    else:
        ws = torch.zeros(system.workspace_size(e.count), dtype=torch.uint8, device="cuda")
        N_.dedup(system, opts, e, ws, lst, cnt)
    torch.cuda.synchronize()
    c = int(cnt.item())
    return (e.tensors["cls"].cpu().numpy(), set(lst[:c].cpu().numpy().tolist()), c)


@pytest.fixture(scope="module")
def tracked():
    """Every path of an N=7 ring tracked in FP64 and certified on the GPU, then planted
    copies of certified endpoints (exact, and moved by 1e-13 relative) in place of 64
    uncertified ones, under higher path indices: 4096 entries, several blocks of every
    dedup kernel.  Returns the index where the copies start."""
    import torch
    N_ = nphc()
    N, sigma, seed = 7, 1.5, 21
    inst = I.ring(N, sigma, seed)
    system = N_.System(N, sigma)
    P = 4 ** (N - 1)
    ep = N_.DeviceEndpoints.empty(2 * (N - 1), np.arange(P))
    opts = N_.options_default(gamma=inst.gamma, precision=N_.PREC_FP64)
    ws = torch.zeros(system.workspace_size(P), dtype=torch.uint8, device="cuda")
    N_.track(system, opts, N_.PREC_FP64, ep, ws)
    N_.refine_certify(system, opts, ep)
    torch.cuda.synchronize()
    cls = ep.tensors["cls"].cpu().numpy()
    cert = np.nonzero(np.isin(cls, [N_.END_REAL, N_.END_NONREAL]))[0]
    assert len(cert) >= 64
    rng = np.random.default_rng(7)
    picks = rng.choice(cert, size=64, replace=False)
    # at most 4^(N-1) entries: 64 uncertified entries make room for the copies
    drop = np.setdiff1d(np.arange(P), cert)[-64:]
    idx = np.concatenate([np.setdiff1d(np.arange(P), drop), picks])
    planted = _select(N_, ep, idx, np.arange(P))
    zr, zi = planted.tensors["z_re"], planted.tensors["z_im"]
    zr[:, P - 32:] *= (1 + 1e-13)
    zi[:, P - 32:] *= (1 + 1e-13)
    return N_, system, opts, planted, P - 64


def test_noalloc_dedup_matches_workspace_dedup_twice(tracked):
    N_, system, opts, ep, P = tracked
    ref = _run(N_, system, opts, ep, noalloc=False)
    assert (ref[0][P:] == N_.END_DUPLICATE).all()   # every planted copy is flagged
    assert ref[2] >= 2 * (len(ref[0]) - P)
    for _ in range(2):   # two calls in a row on the shared array
        got = _run(N_, system, opts, ep, noalloc=True)
        assert np.array_equal(got[0], ref[0])
        assert got[1] == ref[1]
        assert got[2] == ref[2]


def test_noalloc_dedup_smaller_set_after_larger(tracked):
    """A smaller call after a larger one: the leftovers of the larger call in the shared
    array must not leak into the result."""
    N_, system, opts, ep, P = tracked
    _run(N_, system, opts, ep, noalloc=True)
    sub = _select(N_, ep, np.arange(P - 1000, P + 64), np.arange(1064))
    ref = _run(N_, system, opts, sub, noalloc=False)
    for _ in range(2):
        got = _run(N_, system, opts, sub, noalloc=True)
        assert np.array_equal(got[0], ref[0])
        assert got[1] == ref[1] and got[2] == ref[2]


def test_empty_set_clears_dup_count():
    """No entries: both entry points still write *dup_count = 0 (the caller's sentinel
    must not survive), whatever an earlier call left in the shared array."""
    import torch
    N_ = nphc()
    system = N_.System(7, 1.5)
    opts = N_.options_default()
    ep = N_.DeviceEndpoints.empty(12, np.arange(0))
    for noalloc in (True, False, True):
        cnt = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
        lst = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        if noalloc:
            N_.dedup_noalloc(system, opts, ep, lst, cnt)
        else:
            ws = torch.zeros(max(1, system.workspace_size(0)), dtype=torch.uint8, device="cuda")
            N_.dedup(system, opts, ep, ws, lst, cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == 0
        assert int(lst.item()) == -7   # the list is not written


def test_noalloc_dedup_rejects_counts_beyond_the_limit():
    import torch
    N_ = nphc()
    system = N_.System(10, 1.0)
    ep = N_.DeviceEndpoints.empty(18, torch.arange(N_.DEDUP_NOALLOC_MAX + 1))
    with pytest.raises(N_.NphcError) as ei:
        N_.dedup_noalloc(system, N_.options_default(), ep)
    assert ei.value.status == 1
    assert "NPHC_DEDUP_NOALLOC_MAX" in str(ei.value)
