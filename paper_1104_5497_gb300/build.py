"""In-tree build of libnphc.so (the CUDA library behind include/nphc.h) for sm_103a.

Every kernel family is instantiated per ring size in its own object so that nvcc runs
in parallel; the objects are linked into paper_1104_5497_gb300/_build/libnphc.so.  A
stamp of the sources and flags skips the build when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnphc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
M_RANGE = range(2, 13)          # N = 3 .. 13
KINDS = {0: "track_f32", 1: "track_f64", 2: "endgame", 3: "cauchy"}
QUAD_RANGE = range(1, 13)       # generic quadratic systems, n = 1 .. 12 unknowns


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnphc")


PEAK_LIB = os.path.join(OUT, "libnphc_peak.so")   # FMA microbenchmark (alu_peak.cu)


def _units():
    units = []
    for f in ("nphc_api.cu", "nphc_kernels.cu", "xy_dispatch.cu"):
        units.append((f, [], f.replace(".cu", ".o")))
    for kind, name in KINDS.items():
        for m in M_RANGE:
            units.append(("xy_inst.cu", [f"-DNPHC_INST_M={m}", f"-DNPHC_INST_KIND={kind}"],
                          f"xy_{name}_m{m}.o"))
    for nv in QUAD_RANGE:
        units.append(("quad_inst.cu", [f"-DNPHC_QUAD_NV={nv}"], f"quad_n{nv}.o"))
    return units


def _stamp() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                h.update(f.encode())
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


DEBUG_OUT = os.path.join(OUT, "debug")
DEBUG_LIB = os.path.join(DEBUG_OUT, "libnphc.so")
DEBUG_FLAGS = ["-DNPHC_DEBUG", "-rdc=true"]   # one error word shared by every unit


def _build_variant(out: str, lib: str, extra: list, peak: bool, force: bool, jobs, verbose) -> str:
    os.makedirs(out, exist_ok=True)
    stamp_file = os.path.join(out, "libnphc.stamp")
    stamp = _stamp() + " ".join(extra)
    if (not force and os.path.exists(lib) and (not peak or os.path.exists(PEAK_LIB))
            and os.path.exists(stamp_file) and open(stamp_file).read() == stamp):
        return lib
    nvcc = _nvcc()
    jobs = jobs or max(1, os.cpu_count() or 1)

    def compile_one(u):
        src, defs, obj = u
        cmd = [nvcc] + ARCH + NVCC_FLAGS + extra + defs + ["-c", os.path.join(CSRC, src),
                                                           "-o", os.path.join(out, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {defs}:\n{r.stderr}")
        if verbose:
            print("built", obj, flush=True)
        return os.path.join(out, obj)

    units = _units() + ([("alu_peak.cu", [], "alu_peak.o")] if peak else [])
    # the biggest instantiations first so the pool's tail is short
    units.sort(key=lambda u: -int(u[1][0].split("=")[1]) if u[1] else 0)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(compile_one, units))
    peak_obj = os.path.join(out, "alu_peak.o")
    if peak:
        tmp = PEAK_LIB + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp, peak_obj], capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed (libnphc_peak):\n" + r.stderr)
        os.replace(tmp, PEAK_LIB)
    tmp = lib + f".tmp{os.getpid()}"
    link = [nvcc] + ARCH + [f for f in extra if f.startswith("-rdc")] + ["-shared", "-o", tmp]
    r = subprocess.run(link + [o for o in objs if o != peak_obj], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, lib)
    with open(stamp_file, "w") as fh:
        fh.write(stamp)
    return lib


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile and link libnphc.so (and the FMA microbenchmark's library); returns its path."""
    return _build_variant(OUT, LIB, [], True, force, jobs, verbose)


def build_debug(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """The debug build (NPHC_DEBUG: every kernel checks its work-list, list, dedup-link and
    batch indices, records the first failure for nphc_debug_check and skips the access),
    in _build/debug/; returns its path.  Not part of build(): a test builds it on demand."""
    return _build_variant(DEBUG_OUT, DEBUG_LIB, DEBUG_FLAGS, False, force, jobs, verbose)


if __name__ == "__main__":
    import time
    t0 = time.time()
    print(build(verbose=True), f"{time.time() - t0:.1f}s")
