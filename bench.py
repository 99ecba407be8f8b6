#!/usr/bin/env python3
"""Benchmark: certified paths/s of the NPHC method (arXiv:1104.5497) on one GB300.

Workload: the power-law XY ring N = 10 with sigma ~ U[0.5, 3] and gamma drawn from
seed 2 (inputs.workload_n10): 18 unknowns, 4^9 = 262,144 paths.  One step = the whole
method on every path -- FP32 tracking, FP64 hand-off and re-track, FP64 refinement,
alpha-theory certification, deduplication, Hessian classification -- through
nphc_solve_into on device-resident buffers.  value = paths / step time.

Also reported on the same JSON line:
  e2e           the same metric through the C ABI with host buffers (system built from
                host couplings, nphc_solve allocating and synchronising, stationary
                points and counters copied back), every copy inside the timed region;
  roofline      the FP32 path tracker (the dominant kernel): the method's FP32 flops per
                launch (structured solves and the corrector's residual as a plain
                evaluation; the float-float overhead of the compensated residual reported
                beside it) over its CUDA-event duration, against the FP32 FMA peak measured
                in the same run (csrc/alu_peak.cu); fp64_tail: the FP64 continuation of the
                FP32 pass's hand-offs against the measured FP64 FMA peak;
  cpu_baseline  the CPU oracle on a sample of the same paths, all host cores;
  plain_fp64    the same solve with every step in FP64 (the comparison the metric names);
  clocks        nvidia-smi samples taken during the timed region.

`--impl reference` times the CPU oracle alone on a bounded sample per step.
Multi-GPU (torchrun): every rank solves its own replica of the workload (the method has
no exchange step), value = all ranks' paths / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x lanes x FMA x max clock (context)
METRIC = "certified paths/s at XY N=10 (262k paths), mixed-prec batched vs plain FP64"


# ------------------------------------------------------------------ helpers --
def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest x over all ranks (the slowest replica's time); x itself at world 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(paths_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job paths/s: every rank solves its own replica of the workload."""
    return world * paths_per_rank / seconds


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"nphc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def solve_flops(M: int, corrector: bool) -> tuple[float, float]:
    """FP32 flops of one structured solve of the per-thread tracker as implemented
    (xy_solve.cuh, light-cone coordinates), as (method, overhead).  method: the Schur
    build (couplings sums, -H_t rows, frames, M x M entries and right-hand sides), the
    LU factorisation with partial pivoting, back substitution and recovery; a corrector
    solve adds the second
    right-hand side and the residual -H counted as a plain evaluation.  overhead: what the
    compensated (float-float) residual costs beyond that plain evaluation.  A complex
    product is 6 flops, a complex sum 2, a complex times real 2, |z|^2 3, a square root or
    reciprocal 1; one float-float accumulate is 10 (exact product 2, two-sum 6, two adds),
    12 with a low part."""
    nr = 2 if corrector else 1
    column = M * (42 + 18 * (nr - 1)) + 219
    build = M * column
    lu = 0
    for k in range(M):   # pivot |a|^2, sqrt, complex reciprocal, multipliers, rank-one update
        n = M - k
        lu += 3 * n + 7 + 6 * (n - 1) + (M - 1 - k + nr) * 8 * (n - 1)
    back = sum(6 * nr + 8 * k * nr for k in range(M))
    recover = M * (111 + 42 * (nr - 1))
    method = float(build + lu + back + recover)
    overhead = 0.0
    if corrector:
        method += M * (8 * M + 63)
        overhead = float(M * (32 * M + 421))
    return method, overhead


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1104_5497_gb300", "csrc")
    for f in ("xy_solve.cuh", "xy_track.cuh", "nphc_internal.cuh"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the FP32 tracker from the committed ncu summary, if it was
    taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "xy_track_f32_n10.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    if d.get("kernel_source_sha") != kernel_source_sha():
        return None
    return d.get("dram_bytes_per_launch")


# --------------------------------------------------------------- the oracle --
def oracle_sample_rate(inst, n_paths: int, seed: int = 0, collect: bool = False):
    """Paths/s of the CPU oracle (track, refine, certify, dedup, classify) on a random
    sample of n_paths paths of the workload, in contiguous chunks of 64.  collect: also
    return the sample's path indices, classes and endpoints (a fifth value)."""
    import oracle as O
    J = O.couplings(inst.N, inst.sigma)
    T = O.xy_terms(inst.N, J)
    P = 4 ** (inst.N - 1)
    rng = np.random.default_rng(seed)
    chunks = max(1, n_paths // 64)
    starts = rng.choice(P // 64, size=chunks, replace=False) * 64
    threads = O.default_threads()
    kept = []
    t0 = time.perf_counter()
    for s in starts:
        out = O.solve_system(T, inst.gamma, path0=int(s), npaths=64, nthreads=threads)
        for i in np.nonzero(out["cls"] == O.C_REAL)[0]:
            z = out["z"][i]
            O.xy_classify(inst.N, J, z[:inst.N - 1].real, z[inst.N - 1:].real)
        if collect:
            kept.append((out["path"], out["cls"], out["z"]))
    dt = time.perf_counter() - t0
    if not collect:
        return chunks * 64 / dt, chunks * 64, threads, dt
    sample = {"path": np.concatenate([k[0] for k in kept]), "cls": np.concatenate([k[1] for k in kept]),
              "z": np.concatenate([k[2] for k in kept])}
    return chunks * 64 / dt, chunks * 64, threads, dt, sample


def sample_parity(sample, gpu_cls, gpu_z) -> dict:
    """The GPU solve against the oracle on the oracle's sample of paths: paths certified
    by one and not the other, paths real in one and not the other, and the largest
    endpoint difference (relative to 1 + |z|) over the paths both certify.  The oracle
    deduplicates within each 64-path chunk only, so a GPU duplicate counts as certified.
    Class numbers are shared (NPHC_END_* = the oracle's)."""
    p = np.asarray(sample["path"], dtype=np.int64)
    oc, gc = np.asarray(sample["cls"]), np.asarray(gpu_cls)[p]
    o_cert = np.isin(oc, [2, 3, 4, 5])
    g_cert = np.isin(gc, [2, 3, 4, 5])
    both = o_cert & g_cert
    err = 0.0
    if both.any():
        zo, zg = np.asarray(sample["z"])[both], np.asarray(gpu_z)[p[both]]
        err = float((np.abs(zo - zg).max(axis=1) / (1 + np.abs(zo).max(axis=1))).max())
    return {"paths": int(len(p)), "certified": int(both.sum()),
            "class_mismatches": int((o_cert != g_cert).sum()),
            "real_mismatches": int(((oc == 2) != (gc == 2)).sum()), "max_rel_err": err}


def run_reference(args):
    rank, local, world = env_rank()
    if rank != 0:
        return
    from paper_1104_5497_gb300 import inputs
    inst = inputs.workload_n10()
    for _ in range(args.warmup):
        oracle_sample_rate(inst, args.ref_paths, seed=100)
    rates, secs = [], []
    for k in range(args.steps):
        r, n, cores, dt = oracle_sample_rate(inst, args.ref_paths, seed=k)
        rates.append(r)
        secs.append(dt)
    v = float(np.mean(rates))
    sample = f"{n} of {4 ** 9} paths per step (random 64-path chunks), whole method"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "paths/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(inst),
            "cpu_baseline": {"value": v, "unit": "paths/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(inst):
    return {"workload": "XY power-law ring N=10, sigma~U[0.5,3] (seed 2): 18 unknowns, 262,144 paths",
            "N": inst.N, "sigma": round(inst.sigma, 6), "paths": 4 ** (inst.N - 1),
            "precision": "mixed (FP32 tracking, FP64 hand-off/refine/certify/classify)",
            "l2": "flushed (256 MB write) before every timed step"}


# ------------------------------------------------------------------ our arm --
def run_mine(args):
    import torch
    import paper_1104_5497_gb300.nphc as nphc
    from paper_1104_5497_gb300 import build, inputs

    rank, local, world = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    inst = inputs.workload_n10()
    P = 4 ** (inst.N - 1)
    M = inst.N - 1
    system = nphc.System(inst.N, inst.sigma)
    opts = nphc.options_default(gamma=inst.gamma, precision=nphc.PREC_MIXED)
    opts_default = opts
    tuned = {"autotuned": False}
    if not args.no_autotune:   # per (N, GPU), outside every timed region
        from paper_1104_5497_gb300 import autotune
        # a profiler run launches nothing extra: it takes the cached choice of an earlier
        # run, or the defaults
        opts, rep_ = autotune.tune(system, opts, measure=not args.profile)
        tuned = {"autotuned": True, "cached": rep_["cached"]}
        for k in ("blocks_per_sm", "list_blocks_per_sm", "threads_per_path", "max_newton_fp32",
                  "eps_fp32", "step_gate"):
            if k in rep_:
                tuned[k] = rep_[k]
    res = nphc.Result(system)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # ---- device-resident value
    for _ in range(args.warmup):
        nphc.solve_into(system, opts, res)
    barrier()
    times = []
    with ClockSampler(local) as clk:
        barrier()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            nphc.solve_into(system, opts, res)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier()
    ms = max_over_ranks(float(np.mean(times)), world)
    counts = res.counts()
    if args.profile:
        # profiler captures: the solve loop only, no bench line
        if rank == 0:
            print(json.dumps({"profile": True, "ms_per_step": ms, "steps": args.steps,
                              "warmup": args.warmup, "counts": counts}), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    launches = counts["launches"] * args.steps
    value = replica_value(P, world, ms / 1e3)

    # ---- measured FMA peaks (after the timed solves, so that their heat does not reach them)
    from paper_1104_5497_gb300.peaks import alu_peak
    p32, p64 = alu_peak(32), alu_peak(64)

    def timed(fn):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)

    # ---- the dominant kernel alone: FP32 tracker, CUDA events on the launching stream
    ep = nphc.DeviceEndpoints.empty(2 * M, np.arange(P))
    ws = torch.zeros(system.workspace_size(P), dtype=torch.uint8, device="cuda")
    nphc.track(system, opts, nphc.PREC_MIXED, ep, ws)
    torch.cuda.synchronize()
    kt = [timed(lambda: nphc.track(system, opts, nphc.PREC_MIXED, ep, ws))
          for _ in range(max(3, args.steps))]
    solves = int(ep.tensors["solves"].sum().item())
    newton = int(ep.tensors["newton"].sum().item())
    fp_pred, fp_corr = solve_flops(M, False), solve_flops(M, True)
    flops = (solves - newton) * fp_pred[0] + newton * fp_corr[0]
    eft_flops = newton * fp_corr[1]
    k_ms = float(np.mean(kt))
    achieved = flops / (k_ms / 1e3) / 1e12
    traffic = profiled_traffic()

    # ---- the FP64 continuation of the FP32 pass's hand-offs alone (one path per warp)
    st = ep.tensors["status"]
    hl = torch.nonzero((st == nphc.PATH_HANDOFF) | (st == nphc.PATH_HANDOFF_COND)).flatten().to(torch.int32)
    hn = torch.tensor([hl.numel()], dtype=torch.int32, device="cuda")
    saved = {k: v.clone() for k, v in ep.tensors.items()}

    def restore():
        for k, v in saved.items():
            ep.tensors[k].copy_(v)
    nphc.track(system, opts, nphc.PREC_FP64, ep, ws, hl, hn, resume=True)   # warm
    restore()
    torch.cuda.synchronize()
    t64 = timed(lambda: nphc.track(system, opts, nphc.PREC_FP64, ep, ws, hl, hn, resume=True))
    hidx = hl.long()
    s64 = int((ep.tensors["solves"][hidx] - saved["solves"][hidx]).sum().item())
    n64 = int((ep.tensors["newton"][hidx] - saved["newton"][hidx]).sum().item())
    f64 = (s64 - n64) * fp_pred[0] + n64 * (fp_corr[0] + fp_corr[1])
    del saved

    # ---- the same solve with the library's default options (no autotuning)
    ms_untuned = None
    if tuned["autotuned"]:
        nphc.solve_into(system, opts_default, res)
        ms_untuned = float(np.mean([timed(lambda: nphc.solve_into(system, opts_default, res))
                                    for _ in range(3)]))

    # ---- what the condition test costs: the same solve without it
    import ctypes
    opts_nok = nphc.nphc_options()
    ctypes.memmove(ctypes.byref(opts_nok), ctypes.byref(opts), ctypes.sizeof(opts_nok))
    opts_nok.kappa_fp32 = 0.0
    nphc.solve_into(system, opts_nok, res)
    ms_nok = timed(lambda: nphc.solve_into(system, opts_nok, res))
    nphc.solve_into(system, opts, res)   # leave the result of the benchmarked options
    torch.cuda.synchronize()

    # ---- the N = 12 ring (sigma = 1): 22 unknowns, 4,194,304 paths, same pipeline
    n12 = None
    if not args.no_n12:
        i12 = inputs.workload_n12()
        s12 = nphc.System(i12.N, i12.sigma)
        # the library's default options: the autotuner's calibration sample (262,144 paths)
        # is 6% of this ring, and its scheduling choice measured slower on the whole ring
        o12 = nphc.options_default(gamma=i12.gamma, precision=nphc.PREC_MIXED)
        r12 = nphc.Result(s12)
        nphc.solve_into(s12, o12, r12)
        ms12 = timed(lambda: nphc.solve_into(s12, o12, r12))
        c12 = r12.counts()
        n12 = {"workload": "XY power-law ring N=12, sigma=1 (seed 4): 22 unknowns, 4,194,304 paths",
               "ms_per_step": ms12, "value": 4 ** (i12.N - 1) / (ms12 / 1e3), "unit": "paths/s",
               "real": c12["real"], "nonreal": c12["nonreal"], "singular": c12["singular"],
               "handoff": c12["handoff"], "autotuned": False}
        del r12, s12

    # ---- the 64-ring batch (N = 6..9, per-pair disorder, one gamma each; 1,847,296 paths)
    batch = None
    if not args.no_batch:
        binst = inputs.workload_batch64()
        bsys = [nphc.System(b.N, b.sigma, nphc.xy_couplings(b.N, b.sigma, b.g, b.eps)) for b in binst]
        bopt = [nphc.options_default(gamma=b.gamma, precision=nphc.PREC_MIXED) for b in binst]
        bpaths = sum(x.npaths for x in bsys)
        B = nphc.Batch(bsys)
        bt = {}
        for name, kw in (("grouped", {}), ("grouped_graph", {"graph": True}),
                         ("per_instance", {"per_instance": True})):
            B.solve(bopt, **kw)
            B.solve(bopt, **kw)   # (a graph is captured on the second solve)
            torch.cuda.synchronize()
            bt[name] = timed(lambda: B.solve(bopt, **kw))
        bres = [nphc.Result(x) for x in bsys]

        def singles():
            for x, o, r in zip(bsys, bopt, bres):
                nphc.solve_into(x, o, r)
        singles()
        bt["singles"] = timed(singles)
        batch = {"workload": "64 disordered XY rings, N ~ U{6..9}, sigma ~ U[0.5, 3], J (1 + 0.1 g) per pair (seed 3)",
                 "paths": bpaths, "value": bpaths / (bt["grouped"] / 1e3), "unit": "paths/s",
                 "ms_per_step": bt["grouped"],
                 "mode": "one FP32 launch per ring size over a global (instance, path) queue, eager",
                 "grouped_graph_ms": bt["grouped_graph"], "per_instance_streams_ms": bt["per_instance"],
                 "sum_of_single_solves_ms": bt["singles"]}
        del B, bres

    # ---- plain FP64 on the same workload (the metric's comparison)
    opts64 = nphc.options_default(gamma=inst.gamma, precision=nphc.PREC_FP64,
                                  list_blocks_per_sm=opts.list_blocks_per_sm)
    res64 = nphc.Result(system)
    nphc.solve_into(system, opts64, res64)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    flush.zero_()
    e0.record()
    nphc.solve_into(system, opts64, res64)
    e1.record()
    e1.synchronize()
    ms64 = e0.elapsed_time(e1)
    c64 = res64.counts()
    del res64

    # ---- end to end through the C ABI with host buffers
    J_host = nphc.xy_couplings(inst.N, inst.sigma)

    def e2e(o):
        ts, d2h = [], 0
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = nphc.System(inst.N, inst.sigma, J_host)
            r2 = nphc.solve(s2, o)
            sps = r2.stationary_points()
            r2.counts()
            del r2, s2
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(time.perf_counter() - t0)
            d2h = sum(v.nbytes for v in sps.values()) + 8 * nphc.NCOUNTS
        return max_over_ranks(float(np.mean(ts)), world), d2h
    e2e_s, d2h = e2e(opts)
    e2e_untuned = e2e(opts_default)[0] if tuned["autotuned"] else None

    # ---- CPU oracle on a sample of the same workload (rank 0, N = 1 only)
    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu:
        r, n, cores, dt, sample = oracle_sample_rate(inst, args.cpu_paths, collect=True)
        try:   # the timed solve's endpoints against the oracle on the same sample of paths
            ep_all = res.endpoints()
            parity = sample_parity(sample, ep_all["cls"], ep_all["z"])
        except Exception as exc:   # a report, never a reason to lose the bench line
            parity = {"error": repr(exc)}
        cpu = {"value": r, "unit": "paths/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} of {P} paths (random 64-path chunks), whole method, {dt:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": dict(workload_config(inst), launch=tuned),
                "certified": {"real": counts["real"], "nonreal": counts["nonreal"],
                              "index_hist": counts["index_hist"],
                              "equal_to_plain_fp64": (counts["real"] == c64["real"]
                                                      and counts["nonreal"] == c64["nonreal"]
                                                      and counts["index_hist"] == c64["index_hist"])},
                "plain_fp64": {"value": P / (ms64 / 1e3), "unit": "paths/s", "ms_per_step": ms64,
                               "speedup_mixed_over_fp64": ms64 / ms},
                "certified_per_s": {"solutions": (counts["real"] + counts["nonreal"]) / (ms / 1e3),
                                    "real_sps": counts["real"] / (ms / 1e3)},
                "e2e": {"value": replica_value(P, world, e2e_s), "unit": "paths/s",
                        "h2d_bytes_per_step": int(J_host.nbytes), "d2h_bytes_per_step": int(d2h),
                        "untuned_value": (replica_value(P, world, e2e_untuned)
                                          if e2e_untuned else None)},
                "untuned_ms_per_step": ms_untuned,
                "roofline": {"bound": "alu", "kernel": "xy_track_kernel<9,float> (FP32 tracker)",
                             "achieved": achieved, "peak": p32["tflops"], "unit": "TFLOP/s",
                             "frac": achieved / p32["tflops"],
                             "peak_note": "measured in this run: FP32 FMA microbenchmark (csrc/alu_peak.cu), "
                                          f"nominal {NOMINAL_FP32_TFLOPS:.1f}",
                             "kernel_ms": k_ms, "flops_per_launch": flops,
                             "flop_count": "method only: structured solves + plain residual evaluation",
                             "eft_overhead_flops_per_launch": eft_flops,
                             "frac_with_eft_overhead": (flops + eft_flops) / (k_ms / 1e3) / 1e12 / p32["tflops"],
                             "traffic": traffic},
                "fp64_tail": {"kernel": "xy_track_warp64_kernel<9,4> (FP64 continuation of hand-offs)",
                              "handoffs": int(hl.numel()), "ms": t64, "solves": s64,
                              "achieved_tflops": f64 / (t64 / 1e3) / 1e12 if t64 > 0 else None,
                              "peak_tflops": p64["tflops"], "peak_note": "measured FP64 FMA microbenchmark",
                              "frac": (f64 / (t64 / 1e3) / 1e12) / p64["tflops"] if t64 > 0 else None},
                "condition_test": {"kappa_fp32": opts.kappa_fp32, "handoffs": counts["handoff_cond"],
                                   "ms_per_step_without": ms_nok},
                "alu_peaks": {"fp32_tflops": p32["tflops"], "fp64_tflops": p64["tflops"]},
                "n12": n12,
                "batch64": batch,
                "cpu_baseline": cpu,
                "oracle_parity": parity,
                "gpu_launches": launches,
                "clocks": clk.summary(),
                "counts": {k: v for k, v in counts.items() if k != "index_hist"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--cpu-paths", type=int, default=8192, help="oracle sample for cpu_baseline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="the library's default options instead of the autotuned ones")
    ap.add_argument("--ref-paths", type=int, default=2048, help="oracle sample per reference step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-n12", action="store_true", help="skip the N = 12 solve")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-ring batch")
    ap.add_argument("--profile", action="store_true",
                    help="run only the timed solve loop (for profiler captures); no bench line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
