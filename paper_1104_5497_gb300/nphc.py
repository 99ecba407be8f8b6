"""Python binding of libnphc (include/nphc.h): the same calls, argument marshalling only.

Every step of the method runs in the CUDA library; PyTorch only provides device memory
and streams.  There is no CPU fallback: loading fails loudly when the library is
missing, and the compute calls raise when no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnphc.so")

NPHC_MIN_N, NPHC_MAX_N = 3, 13
PREC_FP64, PREC_MIXED = 0, 1

PATH_RUNNING, PATH_REACHED, PATH_DIVERGED, PATH_MIN_STEP, PATH_STEP_BUDGET, PATH_NONFINITE, \
    PATH_HANDOFF, PATH_HANDOFF_COND = range(8)
END_NONE, END_SINGULAR, END_REAL, END_NONREAL, END_UNDECIDED, END_DUPLICATE, END_FAILED = range(7)

COUNT_NAMES = ["paths", "reached", "diverged", "failed", "real", "nonreal", "undecided",
               "singular", "duplicate", "handoff", "retracked", "solves", "launches"]
# after the index histogram (NPHC_COUNT_EG_*, then NPHC_COUNT_HANDOFF_COND)
EG_COUNT_NAMES = ["eg_run", "eg_converged", "eg_multiple", "eg_at_infinity"]
TAIL_COUNT_NAMES = ["handoff_cond"]
NCOUNTS = len(COUNT_NAMES) + NPHC_MAX_N + len(EG_COUNT_NAMES) + len(TAIL_COUNT_NAMES)
# Cauchy endgame outcomes (NPHC_EG_*)
EG_NONE, EG_CONVERGED, EG_NOT_CLOSED, EG_NOT_CONVERGED, EG_TRACK_FAILED, EG_DIVERGED, \
    EG_AT_INFINITY = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EBUDGET", 5: "ESTATE"}
BATCH_GRAPH, BATCH_PER_INSTANCE = 1, 2   # nphc_batch_solve flags


class NphcError(RuntimeError):
    def __init__(self, call: str, status: int, msg: str):
        super().__init__(f"{call}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class nphc_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int),
                ("gamma_re", ctypes.c_double), ("gamma_im", ctypes.c_double),
                ("tol_sol", ctypes.c_double), ("tol_real", ctypes.c_double),
                ("h0", ctypes.c_double), ("h_max", ctypes.c_double), ("h_min", ctypes.c_double),
                ("eps_fp32", ctypes.c_double), ("eps_fp64", ctypes.c_double),
                ("trust", ctypes.c_double), ("trust_fp32", ctypes.c_double),
                ("r_div", ctypes.c_double),
                ("max_newton_fp32", ctypes.c_int), ("max_newton_fp64", ctypes.c_int),
                ("max_steps", ctypes.c_int), ("max_steps_fp32", ctypes.c_int),
                ("crawl_steps_fp32", ctypes.c_int),
                ("grow_after", ctypes.c_int),
                ("refine_iters", ctypes.c_int), ("refine_eps", ctypes.c_double),
                ("block_size", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("endgame", ctypes.c_int), ("eg_r0", ctypes.c_double),
                ("eg_ratio", ctypes.c_double), ("eg_radii", ctypes.c_int),
                ("eg_samples", ctypes.c_int), ("eg_max_cycle", ctypes.c_int),
                ("eg_tol_close", ctypes.c_double), ("eg_tol_conv", ctypes.c_double),
                ("eg_h_min", ctypes.c_double), ("eg_max_attempts", ctypes.c_int),
                ("list_blocks_per_sm", ctypes.c_int),
                ("kappa_sing", ctypes.c_double), ("threads_per_path", ctypes.c_int),
                ("kappa_fp32", ctypes.c_double)]


_P = ctypes.c_void_p


class nphc_endpoints(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("path", _P), ("z_re", _P), ("z_im", _P),
                ("t", _P), ("h", _P), ("status", _P), ("steps", _P), ("solves", _P),
                ("newton", _P), ("cls", _P), ("alpha", _P), ("beta", _P), ("gamma", _P),
                ("resid", _P)]


_lib = None


def use_library(path: str) -> None:
    """Load the library from `path` (e.g. the debug build) instead of the default; must
    come before the first call that loads it."""
    global LIB_PATH
    if _lib is not None:
        raise RuntimeError("libnphc is already loaded")
    LIB_PATH = path


def lib():
    """Load libnphc.so (built by paper_1104_5497_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnphc.so not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, d, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    pd, pi64 = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    pi32 = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "nphc_options_default": [ctypes.POINTER(nphc_options)],
        "nphc_xy_couplings": [i32, d, pd, d, pd],
        "nphc_xy_couplings_vjp": [i32, d, pd, d, pd, pd],
        "nphc_system_create_xy": [i32, d, pd, ctypes.POINTER(vp)],
        "nphc_system_create_quadratic": [i32, i32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32), pd, pd,
                                         ctypes.POINTER(vp)],
        "nphc_system_info": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), pi64],
        "nphc_system_couplings": [vp, pd],
        "nphc_workspace_size": [vp, i64, ctypes.POINTER(ctypes.c_size_t)],
        "nphc_track": [vp, ctypes.POINTER(nphc_options), i32, ctypes.POINTER(nphc_endpoints),
                       vp, vp, i32, vp, ctypes.c_size_t, vp],
        "nphc_refine_certify": [vp, ctypes.POINTER(nphc_options), ctypes.POINTER(nphc_endpoints),
                                vp, vp, vp],
        "nphc_endgame": [vp, ctypes.POINTER(nphc_options), ctypes.POINTER(nphc_endpoints), vp, vp,
                         vp, vp, vp, ctypes.c_size_t, vp],
        "nphc_result_copy_endgame": [vp, i64, pi32, pi32, pi64],
        "nphc_dedup": [vp, ctypes.POINTER(nphc_options), ctypes.POINTER(nphc_endpoints), vp, vp,
                       vp, ctypes.c_size_t, vp],
        "nphc_dedup_noalloc": [vp, ctypes.POINTER(nphc_options), ctypes.POINTER(nphc_endpoints),
                               vp, vp, vp],
        "nphc_classify": [vp, ctypes.POINTER(nphc_endpoints), vp, vp, vp, vp, vp, vp],
        "nphc_result_create": [vp, ctypes.POINTER(vp)],
        "nphc_solve_into": [vp, ctypes.POINTER(nphc_options), vp, vp],
        "nphc_solve": [vp, ctypes.POINTER(nphc_options), vp, ctypes.POINTER(vp)],
        "nphc_result_counts": [vp, pi64],
        "nphc_result_copy_sps": [vp, i64, pd, pd, pi32, pd, pi64, pd, pi64],
        "nphc_result_copy_endpoints": [vp, i64, pd, pd, pi32, pi32, pi64],
        "nphc_result_endpoints": [vp, ctypes.POINTER(nphc_endpoints)],
        "nphc_xy_adjoint": [vp, i64, vp, vp, vp, vp, vp],
        "nphc_batch_create": [i32, ctypes.POINTER(vp), ctypes.POINTER(vp)],
        "nphc_batch_solve": [vp, ctypes.POINTER(nphc_options), i32, vp],
        "nphc_batch_result": [vp, i32, ctypes.POINTER(vp)],
        "nphc_debug_check": [pi32],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.nphc_system_destroy.argtypes = [vp]
    L.nphc_system_destroy.restype = None
    L.nphc_result_destroy.argtypes = [vp]
    L.nphc_result_destroy.restype = None
    L.nphc_batch_destroy.argtypes = [vp]
    L.nphc_batch_destroy.restype = None
    L.nphc_last_error.argtypes = []
    L.nphc_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(call: str, status: int):
    if status != 0:
        raise NphcError(call, status, lib().nphc_last_error().decode())


def _pd(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _pi32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def options_default(**kw) -> nphc_options:
    o = nphc_options()
    _check("nphc_options_default", lib().nphc_options_default(ctypes.byref(o)))
    fields = {f[0] for f in nphc_options._fields_}
    for k, v in kw.items():
        if k == "gamma":
            o.gamma_re, o.gamma_im = float(np.real(v)), float(np.imag(v))
        elif k in fields:
            setattr(o, k, v)
        else:
            raise TypeError(f"nphc_options has no field {k!r}")
    return o


def xy_couplings(N: int, sigma: float, g: np.ndarray | None = None, eps: float = 0.1) -> np.ndarray:
    J = np.zeros((N, N))
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    _check("nphc_xy_couplings", lib().nphc_xy_couplings(int(N), float(sigma),
                                                       None if gg is None else _pd(gg),
                                                       float(eps), _pd(J)))
    return J


def xy_couplings_vjp(N: int, sigma: float, dL_dJ: np.ndarray, g: np.ndarray | None = None,
                     eps: float = 0.1) -> float:
    """nphc_xy_couplings_vjp: dL/dsigma from dL/dJ (N x N) of the couplings."""
    dJ = np.ascontiguousarray(dL_dJ, dtype=np.float64)
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    out = ctypes.c_double()
    _check("nphc_xy_couplings_vjp", lib().nphc_xy_couplings_vjp(int(N), float(sigma),
                                                               None if gg is None else _pd(gg),
                                                               float(eps), _pd(dJ),
                                                               ctypes.byref(out)))
    return out.value


class System:
    """nphc_system: the polynomial system of one XY ring (host-side handle)."""

    def __init__(self, N: int, sigma: float = 1.0, J: np.ndarray | None = None):
        h = ctypes.c_void_p()
        Jc = None if J is None else np.ascontiguousarray(J, dtype=np.float64)
        _check("nphc_system_create_xy",
               lib().nphc_system_create_xy(int(N), float(sigma), None if Jc is None else _pd(Jc),
                                           ctypes.byref(h)))
        self._attach(h)

    def _attach(self, h):
        self.handle = h
        n = ctypes.c_int()
        NN = ctypes.c_int()
        P = ctypes.c_int64()
        _check("nphc_system_info", lib().nphc_system_info(h, ctypes.byref(NN), ctypes.byref(n),
                                                        ctypes.byref(P)))
        self.N, self.n, self.npaths = NN.value, n.value, P.value
        self.M = max(self.N - 1, 0)

    @classmethod
    def quadratic(cls, n: int, eq, va, vb, coef) -> "System":
        """nphc_system_create_quadratic: P_i = sum over terms with eq == i of
        coef * w(va) * w(vb), w(-1) = 1 (a term list, as oracle.Terms)."""
        eq = np.ascontiguousarray(eq, dtype=np.int32)
        va = np.ascontiguousarray(va, dtype=np.int32)
        vb = np.ascontiguousarray(vb, dtype=np.int32)
        coef = np.asarray(coef, dtype=complex)
        cre = np.ascontiguousarray(coef.real, dtype=np.float64)
        cim = np.ascontiguousarray(coef.imag, dtype=np.float64)
        pi32 = ctypes.POINTER(ctypes.c_int32)
        h = ctypes.c_void_p()
        _check("nphc_system_create_quadratic", lib().nphc_system_create_quadratic(
            int(n), int(len(eq)), eq.ctypes.data_as(pi32), va.ctypes.data_as(pi32),
            vb.ctypes.data_as(pi32), _pd(cre), _pd(cim), ctypes.byref(h)))
        self = cls.__new__(cls)
        self._attach(h)
        return self

    def couplings(self) -> np.ndarray:
        J = np.zeros((self.N, self.N))
        _check("nphc_system_couplings", lib().nphc_system_couplings(self.handle, _pd(J)))
        return J

    def workspace_size(self, count: int) -> int:
        b = ctypes.c_size_t()
        _check("nphc_workspace_size", lib().nphc_workspace_size(self.handle, int(count), ctypes.byref(b)))
        return b.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.nphc_system_destroy(self.handle)
            self.handle = None


class Result:
    """nphc_result: device buffers for every path of a system."""

    def __init__(self, system: System):
        h = ctypes.c_void_p()
        _check("nphc_result_create", lib().nphc_result_create(system.handle, ctypes.byref(h)))
        self.handle = h
        self.system = system

    def counts(self) -> dict:
        c = np.zeros(NCOUNTS, np.int64)
        _check("nphc_result_counts", lib().nphc_result_counts(self.handle, _pi64(c)))
        out = {k: int(c[i]) for i, k in enumerate(COUNT_NAMES)}
        out["index_hist"] = [int(v) for v in c[len(COUNT_NAMES):len(COUNT_NAMES) + self.system.M + 1]]
        base = len(COUNT_NAMES) + NPHC_MAX_N
        out.update({k: int(c[base + i]) for i, k in enumerate(EG_COUNT_NAMES)})
        base += len(EG_COUNT_NAMES)
        out.update({k: int(c[base + i]) for i, k in enumerate(TAIL_COUNT_NAMES)})
        return out

    def endgame(self) -> dict:
        """Per path: Cauchy endgame cycle number and status (EG_NONE where it did not run)."""
        P = self.system.npaths
        n = ctypes.c_int64()
        cy, st = np.zeros(P, np.int32), np.zeros(P, np.int32)
        _check("nphc_result_copy_endgame", lib().nphc_result_copy_endgame(
            self.handle, P, _pi32(cy), _pi32(st), ctypes.byref(n)))
        return dict(cycle=cy, status=st)

    def stationary_points(self) -> dict:
        M = self.system.M
        n = ctypes.c_int64()
        _check("nphc_result_copy_sps", lib().nphc_result_copy_sps(self.handle, 0, None, None, None,
                                                                  None, None, None, ctypes.byref(n)))
        k = n.value
        th, en, al, ld = np.zeros((k, M)), np.zeros(k), np.zeros(k), np.zeros(k)
        ix, pa = np.zeros(k, np.int32), np.zeros(k, np.int64)
        _check("nphc_result_copy_sps", lib().nphc_result_copy_sps(self.handle, k, _pd(th), _pd(en),
                                                                  _pi32(ix), _pd(al), _pi64(pa),
                                                                  _pd(ld), ctypes.byref(n)))
        return dict(theta=th, energy=en, index=ix, alpha=al, path=pa, log_abs_det=ld)

    def endpoints(self) -> dict:
        s = self.system
        n = ctypes.c_int64()
        P = s.npaths
        zr, zi = np.zeros((P, s.n)), np.zeros((P, s.n))
        st, cl = np.zeros(P, np.int32), np.zeros(P, np.int32)
        _check("nphc_result_copy_endpoints", lib().nphc_result_copy_endpoints(
            self.handle, P, _pd(zr), _pd(zi), _pi32(st), _pi32(cl), ctypes.byref(n)))
        return dict(z=zr + 1j * zi, status=st, cls=cl)

    def device_endpoints(self) -> nphc_endpoints:
        ep = nphc_endpoints()
        _check("nphc_result_endpoints", lib().nphc_result_endpoints(self.handle, ctypes.byref(ep)))
        return ep

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None and not getattr(self, "borrowed", False):
            _lib.nphc_result_destroy(self.handle)
        self.handle = None


class Batch:
    """nphc_batch: independent systems solved together (one result per instance)."""

    def __init__(self, systems):
        self.systems = list(systems)   # the batch borrows them
        arr = (ctypes.c_void_p * len(self.systems))(*[s.handle.value for s in self.systems])
        h = ctypes.c_void_p()
        _check("nphc_batch_create", lib().nphc_batch_create(len(self.systems), arr, ctypes.byref(h)))
        self.handle = h

    def solve(self, opts, graph: bool = False, per_instance: bool = False, stream=None) -> None:
        """nphc_batch_solve: opts is one nphc_options per instance; graph captures / replays a
        CUDA graph (NPHC_BATCH_GRAPH); per_instance runs every instance's whole solve on its
        stream instead of one FP32 launch per ring size (NPHC_BATCH_PER_INSTANCE)."""
        arr = (nphc_options * len(self.systems))(*opts)
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_PER_INSTANCE if per_instance else 0)
        _check("nphc_batch_solve", lib().nphc_batch_solve(self.handle, arr, flags,
                                                         _stream_ptr(stream)))

    def result(self, i: int) -> Result:
        h = ctypes.c_void_p()
        _check("nphc_batch_result", lib().nphc_batch_result(self.handle, int(i), ctypes.byref(h)))
        r = Result.__new__(Result)
        r.handle = h
        r.system = self.systems[i]
        r.borrowed = True
        r.owner = self
        return r

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.nphc_batch_destroy(self.handle)
        self.handle = None


def debug_check() -> int:
    """nphc_debug_check: the debug build's first failed index check since the last call
    (0 none; -1 for a release build), cleared."""
    c = np.zeros(1, np.int32)
    _check("nphc_debug_check", lib().nphc_debug_check(_pi32(c)))
    return int(c[0])


def solve_into(system: System, opts: nphc_options, result: Result, stream=None) -> None:
    """Asynchronous whole-method solve into an existing result (no allocation)."""
    _check("nphc_solve_into", lib().nphc_solve_into(system.handle, ctypes.byref(opts),
                                                   result.handle, _stream_ptr(stream)))


def solve(system: System, opts: nphc_options, stream=None) -> Result:
    """nphc_solve: allocate, solve, synchronise."""
    h = ctypes.c_void_p()
    _check("nphc_solve", lib().nphc_solve(system.handle, ctypes.byref(opts), _stream_ptr(stream),
                                         ctypes.byref(h)))
    r = Result.__new__(Result)
    r.handle = h
    r.system = system
    return r


# ------------------------------------------------------------ step-by-step --
@dataclass
class DeviceEndpoints:
    """Caller-owned device endpoint arrays (torch tensors) for the step-by-step calls."""
    count: int
    n: int
    tensors: dict

    @classmethod
    def empty(cls, n: int, paths, device="cuda"):
        import torch
        paths = torch.as_tensor(paths, dtype=torch.int64, device=device).contiguous()
        c = int(paths.numel())
        f64 = dict(dtype=torch.float64, device=device)
        i32 = dict(dtype=torch.int32, device=device)
        t = dict(path=paths, z_re=torch.zeros(n, c, **f64), z_im=torch.zeros(n, c, **f64),
                 t=torch.zeros(c, **f64), h=torch.zeros(c, **f64), status=torch.zeros(c, **i32),
                 steps=torch.zeros(c, **i32), solves=torch.zeros(c, **i32),
                 newton=torch.zeros(c, **i32), cls=torch.zeros(c, **i32),
                 alpha=torch.zeros(c, **f64), beta=torch.zeros(c, **f64),
                 gamma=torch.zeros(c, **f64), resid=torch.zeros(c, **f64))
        return cls(c, n, t)

    def struct(self) -> nphc_endpoints:
        ep = nphc_endpoints()
        ep.count = self.count
        for k, v in self.tensors.items():
            setattr(ep, k, v.data_ptr())
        return ep


def track(system: System, opts: nphc_options, prec: int, ep: DeviceEndpoints, workspace,
          list_=None, list_count=None, resume: bool = False, stream=None) -> None:
    s = ep.struct()
    _check("nphc_track", lib().nphc_track(
        system.handle, ctypes.byref(opts), int(prec), ctypes.byref(s),
        None if list_ is None else list_.data_ptr(),
        None if list_count is None else list_count.data_ptr(), int(resume),
        workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream_ptr(stream)))


def refine_certify(system: System, opts: nphc_options, ep: DeviceEndpoints, list_=None,
                   list_count=None, stream=None) -> None:
    s = ep.struct()
    _check("nphc_refine_certify", lib().nphc_refine_certify(
        system.handle, ctypes.byref(opts), ctypes.byref(s),
        None if list_ is None else list_.data_ptr(),
        None if list_count is None else list_count.data_ptr(), _stream_ptr(stream)))


def endgame(system: System, opts: nphc_options, ep: DeviceEndpoints, workspace, cycle, eg_status,
            list_=None, list_count=None, stream=None) -> None:
    """nphc_endgame: FP64 tracking of the selected entries to t = 1 - eg_r0, then the Cauchy
    endgame; writes z (estimates), cycle and eg_status (int32 device tensors [count])."""
    s = ep.struct()
    _check("nphc_endgame", lib().nphc_endgame(
        system.handle, ctypes.byref(opts), ctypes.byref(s),
        None if list_ is None else list_.data_ptr(),
        None if list_count is None else list_count.data_ptr(), cycle.data_ptr(),
        eg_status.data_ptr(), workspace.data_ptr(), workspace.numel() * workspace.element_size(),
        _stream_ptr(stream)))


def dedup(system: System, opts: nphc_options, ep: DeviceEndpoints, workspace, dup_list=None,
          dup_count=None, stream=None) -> None:
    s = ep.struct()
    _check("nphc_dedup", lib().nphc_dedup(
        system.handle, ctypes.byref(opts), ctypes.byref(s),
        None if dup_list is None else dup_list.data_ptr(),
        None if dup_count is None else dup_count.data_ptr(),
        workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream_ptr(stream)))


DEDUP_NOALLOC_MAX = 65536   # NPHC_DEDUP_NOALLOC_MAX
QUAD_MAX_N = 12             # NPHC_QUAD_MAX_N


def dedup_noalloc(system: System, opts: nphc_options, ep: DeviceEndpoints, dup_list=None,
                  dup_count=None, stream=None) -> None:
    """nphc_dedup_noalloc: dedup with the library's fixed scratch array (no workspace)."""
    s = ep.struct()
    _check("nphc_dedup_noalloc", lib().nphc_dedup_noalloc(
        system.handle, ctypes.byref(opts), ctypes.byref(s),
        None if dup_list is None else dup_list.data_ptr(),
        None if dup_count is None else dup_count.data_ptr(), _stream_ptr(stream)))


def classify(system: System, ep: DeviceEndpoints, theta, index, energy, min_abs_eig=None,
             log_abs_det=None, stream=None) -> None:
    s = ep.struct()
    _check("nphc_classify", lib().nphc_classify(
        system.handle, ctypes.byref(s), theta.data_ptr(), index.data_ptr(), energy.data_ptr(),
        None if min_abs_eig is None else min_abs_eig.data_ptr(),
        None if log_abs_det is None else log_abs_det.data_ptr(), _stream_ptr(stream)))


def xy_adjoint(system: System, theta, g_energy=None, g_theta=None, dJ=None, stream=None):
    """nphc_xy_adjoint on device tensors: theta [count, N-1], g_energy [count],
    g_theta [count, N-1] (float64, cuda).  Returns dJ [N, N] (accumulated into dJ if given)."""
    import torch
    if dJ is None:
        dJ = torch.zeros(system.N, system.N, dtype=torch.float64, device=theta.device)
    theta = theta.contiguous()
    ge = None if g_energy is None else g_energy.contiguous()
    gt = None if g_theta is None else g_theta.contiguous()
    _check("nphc_xy_adjoint", lib().nphc_xy_adjoint(
        system.handle, int(theta.shape[0]), theta.data_ptr(),
        None if ge is None else ge.data_ptr(), None if gt is None else gt.data_ptr(),
        dJ.data_ptr(), _stream_ptr(stream)))
    return dJ

