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
  roofline      the FP32 path tracker (the dominant kernel): algorithmic FP32 flops per
                launch over its CUDA-event duration, against the FP32 peak derived from
                152 SMs x 128 lanes x 2 flops x 2.07 GHz;
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

PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # derived: SMs x lanes x FMA x max clock
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


def solve_flops(M: int, corrector: bool) -> float:
    """Algorithmic FP32 flops of one structured solve as implemented (xy_solve.cuh):
    Schur build, Householder QR, back substitution, recovery; the corrector adds the
    second right-hand side and the compensated residual.  FMA = 2 flops; the error-free
    transformations of the compensated residual are counted operation by operation
    (two-product 3, two-sum 6, one float-float accumulate 11, with a low part 13)."""
    Mf = float(M)
    build = Mf * (43 * Mf + 115)
    r = np.arange(M)
    qr = float((16 * r * r + 34 * r + 24).sum())
    back = 8 * Mf * (Mf - 1) / 2 + 3 * Mf
    recover = 81 * Mf
    f = build + qr + back + recover
    if corrector:
        f += Mf * (18 * Mf + 30) + float((16 * r + 8).sum()) + back + 34 * Mf
        f += Mf * (44 * Mf + 376)   # compensated residual
    return f


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
    tuned = {"autotuned": False}
    if args.autotune:   # launch shapes per (N, GPU), outside every timed region
        from paper_1104_5497_gb300 import autotune
        # a profiler run launches nothing extra: it takes the cached shapes of an earlier
        # run, or the defaults
        opts, rep_ = autotune.tune(system, opts, measure=not args.profile)
        tuned = {"autotuned": True, "blocks_per_sm": rep_["blocks_per_sm"],
                 "list_blocks_per_sm": rep_["list_blocks_per_sm"], "cached": rep_["cached"]}
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

    # ---- the dominant kernel alone: FP32 tracker, CUDA events on the launching stream
    ep = nphc.DeviceEndpoints.empty(2 * M, np.arange(P))
    ws = torch.zeros(system.workspace_size(P), dtype=torch.uint8, device="cuda")
    nphc.track(system, opts, nphc.PREC_MIXED, ep, ws)
    torch.cuda.synchronize()
    kt = []
    for _ in range(max(3, args.steps)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        nphc.track(system, opts, nphc.PREC_MIXED, ep, ws)
        e1.record()
        e1.synchronize()
        kt.append(e0.elapsed_time(e1))
    solves = int(ep.tensors["solves"].sum().item())
    newton = int(ep.tensors["newton"].sum().item())
    flops = (solves - newton) * solve_flops(M, False) + newton * solve_flops(M, True)
    k_ms = float(np.mean(kt))
    achieved = flops / (k_ms / 1e3) / 1e12
    traffic = profiled_traffic()

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
    e2e_t, d2h = [], 0
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = nphc.System(inst.N, inst.sigma, J_host)
        r2 = nphc.solve(s2, opts)
        sps = r2.stationary_points()
        c2 = r2.counts()
        del r2, s2
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
        d2h = sum(v.nbytes for v in sps.values()) + 8 * nphc.NCOUNTS
    e2e_s = max_over_ranks(float(np.mean(e2e_t)), world)

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
                "e2e": {"value": replica_value(P, world, e2e_s), "unit": "paths/s",
                        "h2d_bytes_per_step": int(J_host.nbytes), "d2h_bytes_per_step": int(d2h)},
                "roofline": {"bound": "alu", "kernel": "xy_track_kernel<9,float> (FP32 tracker)",
                             "achieved": achieved, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                             "frac": achieved / PEAK_FP32_TFLOPS,
                             "peak_note": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz",
                             "kernel_ms": k_ms, "flops_per_launch": flops,
                             "traffic": traffic},
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
    ap.add_argument("--autotune", action="store_true",
                    help="autotuned launch shapes instead of the defaults")
    ap.add_argument("--ref-paths", type=int, default=2048, help="oracle sample per reference step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="run only the timed solve loop (for profiler captures); no bench line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
