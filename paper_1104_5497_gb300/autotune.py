"""Autotuner for the launch shapes of the two tracking kernels, per (ring size, GPU).

It times the kernels on a calibration sample of the ring's own paths: the FP32 tracker over
its resident blocks per SM (`nphc_options.blocks_per_sm`), then the FP64 list tracker over
the sample's hand-offs at 1 to 4 blocks per SM (`list_blocks_per_sm`).  Only knobs that
leave every path's arithmetic unchanged are searched.  A path's computation does not
depend on the thread or SM that runs it, so a tuned solve gives the same endpoints, bit
for bit.  The step-control constants keep their defaults: they decide which paths jump,
and with that the re-tracking work, and the oracle uses the same values.  The result is
cached in a JSON file under a key made of N, the GPU's name and its SM count.

The list tracker's best shape depends on how long the hand-off list is, so the sample
must reproduce it: by default it is every path up to N = 10 (262,144).  On the N = 10
ring a 65,536-path sample (241 hand-offs) preferred one block per SM, which is slower on
the whole ring's 1,565 hand-offs than the default two (186.5 ms against 183.4 ms per
solve).

Every step runs through the C ABI (nphc_track on caller-owned device buffers); this
module only chooses options and times calls with CUDA events.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import nphc as N_

FP32_CANDIDATES = (0, 7, 6, 5, 4)   # resident blocks per SM; 0 = the occupancy maximum
LIST_CANDIDATES = (2, 1, 3, 4)      # blocks of 4 warps per SM (the default, 2, first)
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def calibration_paths(npaths: int, sample: int) -> np.ndarray:
    """`sample` path indices spread evenly over [0, npaths) (all of them if fewer)."""
    if sample >= npaths:
        return np.arange(npaths, dtype=np.int64)
    return (np.arange(sample, dtype=np.int64) * npaths) // sample


def pick(timings: dict) -> int:
    """The fastest candidate; ties go to the one listed first (the default)."""
    best, best_t = None, None
    for k, t in timings.items():
        if best_t is None or t < best_t:
            best, best_t = k, t
    return int(best)


def cache_key(N: int, device_name: str, sms: int) -> str:
    return f"N={N}|{device_name}|sms={sms}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, entry: dict) -> None:
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(opts, entry: dict):
    """A copy of opts with the tuned launch shapes."""
    o = N_.nphc_options()
    ctypes.memmove(ctypes.byref(o), ctypes.byref(opts), ctypes.sizeof(o))
    o.blocks_per_sm = int(entry["blocks_per_sm"])
    o.list_blocks_per_sm = int(entry["list_blocks_per_sm"])
    return o


def _median_ms(fn, reps: int) -> float:
    import torch
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def tune(system, opts, sample: int = 262144, reps: int = 3, cache: str | None = DEFAULT_CACHE,
         refresh: bool = False, measure: bool = True):
    """Returns (tuned options, report).  report: the key, the chosen values, the timings
    (ms per candidate) and whether it came from the cache.  measure=False: the cached
    entry if there is one, else opts unchanged (no kernel launches)."""
    import torch
    if system.N == 0:   # generic quadratic systems: FP64 only, nothing to choose
        return apply(opts, dict(blocks_per_sm=opts.blocks_per_sm,
                                list_blocks_per_sm=opts.list_blocks_per_sm)), dict(cached=False)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    key = cache_key(system.N, props.name, props.multi_processor_count)
    if cache and not refresh:
        hit = load_cache(cache).get(key)
        if hit:
            return apply(opts, hit), dict(hit, key=key, cached=True)
    if not measure:
        same = dict(blocks_per_sm=opts.blocks_per_sm, list_blocks_per_sm=opts.list_blocks_per_sm)
        return apply(opts, same), dict(same, key=key, cached=False)
    paths = calibration_paths(system.npaths, sample)
    ep = N_.DeviceEndpoints.empty(system.n, paths)
    ws = torch.empty(system.workspace_size(ep.count), dtype=torch.uint8, device="cuda")
    # FP32 tracker: every candidate tracks the whole sample from its start points
    fp32 = {}
    for bps in FP32_CANDIDATES:
        o = apply(opts, dict(blocks_per_sm=bps, list_blocks_per_sm=0))
        N_.track(system, o, N_.PREC_MIXED, ep, ws)   # warm-up (kernel attributes, caches)
        fp32[bps] = _median_ms(lambda: N_.track(system, o, N_.PREC_MIXED, ep, ws), reps)
    bps32 = pick(fp32)
    # FP64 list tracker: the sample's hand-offs, continued from the same state each time
    o = apply(opts, dict(blocks_per_sm=bps32, list_blocks_per_sm=0))
    N_.track(system, o, N_.PREC_MIXED, ep, ws)
    torch.cuda.synchronize()
    st = ep.tensors["status"]
    ho = torch.nonzero((st == N_.PATH_HANDOFF) | (st == N_.PATH_HANDOFF_COND)).flatten().to(torch.int32)
    lists = {}
    if ho.numel() > 0:
        count = torch.tensor([ho.numel()], dtype=torch.int32, device="cuda")
        saved = {k: v.clone() for k, v in ep.tensors.items() if k != "path"}

        def restore():
            for k, v in saved.items():
                ep.tensors[k].copy_(v)

        for lb in LIST_CANDIDATES:
            ol = apply(opts, dict(blocks_per_sm=bps32, list_blocks_per_sm=lb))
            run = lambda: N_.track(system, ol, N_.PREC_FP64, ep, ws, ho, count, resume=True)
            restore()
            run()                                      # warm-up
            ts = []
            for _ in range(reps):
                restore()
                torch.cuda.synchronize()
                ts.append(_median_ms(run, 1))
            lists[lb] = float(np.median(ts))
        restore()
    lb = pick(lists) if lists else 0
    entry = dict(blocks_per_sm=bps32, list_blocks_per_sm=lb, sample=int(ep.count),
                 handoffs=int(ho.numel()),
                 fp32_ms={str(k): v for k, v in fp32.items()},
                 list_ms={str(k): v for k, v in lists.items()})
    if cache:
        store_cache(cache, key, entry)
    return apply(opts, entry), dict(entry, key=key, cached=False)
