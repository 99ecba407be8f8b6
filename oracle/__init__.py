"""Plain FP64 CPU oracle for the NPHC method of arXiv:1104.5497.

TEST INFRASTRUCTURE ONLY.  The oracle is what the CUDA library is checked against;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  It shares no code with the CUDA path and never calls it.

The arithmetic lives in ``nphc_oracle.c`` (plain C99, ``double complex``, pthreads
over paths).  This module compiles it with gcc on first use (or when the source is
newer than the library) and marshals numpy arrays through ctypes.  Every step of the
method is in the C file; this file only orders the calls:

    couplings  (section "A First Application": J_ij = d_ij^-sigma on the ring)
    xy_terms   (Eq. alg_dec_XY_model_poly, theta_N pinned to 0)
    track      (gamma-trick total-degree homotopy, predictor-corrector tracking)
    endgame    (Cauchy endgame for singular endpoints: turns around t = 1)
    refine_certify (Newton refinement, Delta_sol, alpha-theory, real / non-real tests)
    dedup      (alpha-theory same/distinct tests between certified endpoints)
    xy_classify (theta = atan2(s, c), Hessian index, energy V, log |det H|)
    xy_adjoint  (gradient of a loss on an SP with respect to the couplings)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nphc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Path statuses and endpoint classes of nphc_oracle.c.
REACHED, DIVERGED, MIN_STEP, STEP_BUDGET, NONFINITE = 1, 2, 3, 4, 5
C_NONE, C_SINGULAR, C_REAL, C_NONREAL, C_UNDECIDED, C_DUPLICATE, C_FAILED = 0, 1, 2, 3, 4, 5, 6

ALPHA0 = (13.0 - 3.0 * math.sqrt(17.0)) / 4.0   # Smale's alpha-theorem constant
# FP64 is a soft alpha test (alphaCertified works in exact arithmetic): certify below
# half the constant, so that rounding cannot carry a near-singular point across it
ALPHA_CERT = 0.5 * ALPHA0


class TrackOpts(ctypes.Structure):
    _fields_ = [("h0", ctypes.c_double), ("h_max", ctypes.c_double),
                ("h_min", ctypes.c_double), ("eps_corr", ctypes.c_double),
                ("trust", ctypes.c_double), ("r_div", ctypes.c_double), ("max_newton", ctypes.c_int),
                ("max_steps", ctypes.c_int), ("grow_after", ctypes.c_int)]


class CertOpts(ctypes.Structure):
    _fields_ = [("tol_sol", ctypes.c_double), ("refine_eps", ctypes.c_double),
                ("refine_iters", ctypes.c_int), ("alpha0", ctypes.c_double),
                ("kappa_sing", ctypes.c_double)]


class EgOpts(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_double), ("ratio", ctypes.c_double), ("n_radii", ctypes.c_int),
                ("samples", ctypes.c_int), ("max_cycle", ctypes.c_int),
                ("tol_close", ctypes.c_double), ("tol_conv", ctypes.c_double),
                ("h_min", ctypes.c_double), ("max_attempts", ctypes.c_int),
                ("tol_res", ctypes.c_double)]


# Cauchy endgame outcomes of nphc_oracle.c.
(EG_CONVERGED, EG_NOT_CLOSED, EG_NOT_CONVERGED, EG_TRACK_FAILED, EG_DIVERGED,
 EG_AT_INFINITY) = 1, 2, 3, 4, 5, 6


def default_eg_opts(**kw) -> EgOpts:
    """Cauchy endgame: turns around t = 1 at |1 - t| = 1/16, 1/64, ... (at most 8 radii),
    16 samples per turn, cycle numbers up to 8; a turn closes within 1e-6 (relative), two
    successive estimates agree within 1e-9 (relative) and the estimate solves P within the
    solution tolerance 1e-10 (relative to max(1, ||z||^2))."""
    o = dict(r0=0.0625, ratio=0.25, n_radii=8, samples=16, max_cycle=8, tol_close=1e-6,
             tol_conv=1e-9, h_min=1.0 / 4096, max_attempts=4000, tol_res=1e-10)
    o.update(kw)
    return EgOpts(**o)


def default_track_opts(**kw) -> TrackOpts:
    """Step control of the oracle tracker (the paper gives none; see the design notes).
    A path goes to infinity when ||z||_inf exceeds r_div = 1e8 before t = 1."""
    o = dict(h0=0.01, h_max=0.05, h_min=1e-14, eps_corr=1e-9, trust=0.1, r_div=1e8,
             max_newton=3, max_steps=5000, grow_after=3)
    o.update(kw)
    return TrackOpts(**o)


def default_cert_opts(**kw) -> CertOpts:
    """Delta_sol = 1e-10 (the paper's solution tolerance), alpha_0 from Smale's theorem,
    singular above a Frobenius condition number of 1e12 max(1, ||z||_inf^2)."""
    o = dict(tol_sol=1e-10, refine_eps=1e-14, refine_iters=8, alpha0=ALPHA_CERT, kappa_sing=1e12)
    o.update(kw)
    return CertOpts(**o)


def build(force: bool = False) -> str:
    """Compile nphc_oracle.c into a shared library (gcc, -O2, IEEE semantics, no FMA
    contraction so that the compensated sums stay exact)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        D, I, I64 = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int64
        L.oracle_lu_solve.argtypes = [ctypes.c_int, D, D, D, D, D, D]
        L.oracle_sym_eig.argtypes = [ctypes.c_int, D, D]
        L.oracle_xy_couplings.argtypes = [ctypes.c_int, ctypes.c_double, D, ctypes.c_double, D]
        L.oracle_xy_terms.argtypes = [ctypes.c_int, D, I, I, I, D, D]
        L.oracle_track.argtypes = [ctypes.c_int, ctypes.c_int, I, I, I, D, D, ctypes.c_double,
                                   ctypes.c_double, ctypes.POINTER(TrackOpts), I64, I64,
                                   ctypes.c_int, D, D, I, I, D]
        L.oracle_endgame.argtypes = [ctypes.c_int, ctypes.c_int, I, I, I, D, D, ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(TrackOpts),
                                     ctypes.POINTER(EgOpts), ctypes.POINTER(ctypes.c_int64), I64,
                                     ctypes.c_int, D, D, I, I, D, D]
        L.oracle_sys_eval_jac.argtypes = [ctypes.c_int, ctypes.c_int, I, I, I, D, D, D, D, D, D, D, D]
        L.oracle_sys_eval_acc.argtypes = [ctypes.c_int, ctypes.c_int, I, I, I, D, D, D, D, D, D]
        L.oracle_d2_norm.argtypes = [ctypes.c_int, ctypes.c_int, I, I, I, D, D]
        L.oracle_d2_norm.restype = ctypes.c_double
        L.oracle_refine_certify.argtypes = [ctypes.c_int, ctypes.c_int, I, I, I, D, D,
                                            ctypes.POINTER(CertOpts), I64, ctypes.c_int, D, D,
                                            I, D, I, D, D, D, D, D]
        L.oracle_dedup.argtypes = [ctypes.c_int, I64, D, D, D, D, I]
        L.oracle_dedup.restype = ctypes.c_int64
        L.oracle_xy_classify.argtypes = [ctypes.c_int, D, D, D, D, I, D, D, D, D]
        L.oracle_xy_adjoint.argtypes = [ctypes.c_int, D, D, ctypes.c_double, D, D]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ------------------------------------------------------------------ linear algebra --
def lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    A = np.asarray(A, dtype=complex)
    b = np.asarray(b, dtype=complex)
    n = A.shape[0]
    are, aim = np.ascontiguousarray(A.real), np.ascontiguousarray(A.imag)
    bre, bim = np.ascontiguousarray(b.real), np.ascontiguousarray(b.imag)
    xre, xim = np.zeros(n), np.zeros(n)
    rc = lib().oracle_lu_solve(n, _d(are), _d(aim), _d(bre), _d(bim), _d(xre), _d(xim))
    if rc:
        raise np.linalg.LinAlgError("singular")
    return xre + 1j * xim


def sym_eig(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    w = np.zeros(A.shape[0])
    lib().oracle_sym_eig(A.shape[0], _d(A), _d(w))
    return np.sort(w)


# ---------------------------------------------------------------------- systems --
class Terms:
    """A quadratic system as a term list: P_i = sum coef * w(a) * w(b), w(-1) = 1."""

    def __init__(self, n, eq, va, vb, coef):
        self.n = int(n)
        self.eq = np.ascontiguousarray(eq, dtype=np.int32)
        self.va = np.ascontiguousarray(va, dtype=np.int32)
        self.vb = np.ascontiguousarray(vb, dtype=np.int32)
        coef = np.asarray(coef, dtype=complex)
        self.cre = np.ascontiguousarray(coef.real)
        self.cim = np.ascontiguousarray(coef.imag)

    @property
    def nterms(self):
        return len(self.eq)

    def args(self):
        return (self.n, self.nterms, _i(self.eq), _i(self.va), _i(self.vb), _d(self.cre), _d(self.cim))

    def d2_norm(self) -> float:
        return lib().oracle_d2_norm(*self.args())

    def eval_acc(self, z: np.ndarray) -> np.ndarray:
        """P(z) with exact products and double-double sums, rounded once."""
        n = self.n
        z = np.asarray(z, dtype=complex)
        zre, zim = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        pre, pim = np.zeros(n), np.zeros(n)
        lib().oracle_sys_eval_acc(*self.args(), _d(zre), _d(zim), _d(pre), _d(pim))
        return pre + 1j * pim

    def eval_jac(self, z: np.ndarray):
        """P(z) and DP(z) of the term list."""
        n = self.n
        z = np.asarray(z, dtype=complex)
        zre, zim = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
        pre, pim, dre, dim = np.zeros(n), np.zeros(n), np.zeros((n, n)), np.zeros((n, n))
        lib().oracle_sys_eval_jac(*self.args(), _d(zre), _d(zim), _d(pre), _d(pim), _d(dre), _d(dim))
        return pre + 1j * pim, dre + 1j * dim


def couplings(N: int, sigma: float, g: np.ndarray | None = None, eps: float = 0.1) -> np.ndarray:
    J = np.zeros((N, N))
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    rc = lib().oracle_xy_couplings(N, float(sigma), None if gg is None else _d(gg), float(eps), _d(J))
    if rc:
        raise ValueError("invalid N")
    return J


def xy_terms(N: int, J: np.ndarray) -> Terms:
    m = N - 1
    cap = 2 * m * (N - 1) + 3 * m
    eq, va, vb = (np.zeros(cap, np.int32) for _ in range(3))
    cre, cim = np.zeros(cap), np.zeros(cap)
    Jc = np.ascontiguousarray(J, dtype=np.float64)
    nt = lib().oracle_xy_terms(N, _d(Jc), _i(eq), _i(va), _i(vb), _d(cre), _d(cim))
    return Terms(2 * m, eq[:nt], va[:nt], vb[:nt], cre[:nt] + 1j * cim[:nt])


# --------------------------------------------------------------------- pipeline --
def track(T: Terms, gamma: complex, path0: int = 0, npaths: int | None = None,
          opts: TrackOpts | None = None, nthreads: int | None = None) -> dict:
    n = T.n
    if npaths is None:
        npaths = (1 << n) - path0
    opts = opts or default_track_opts()
    nthreads = nthreads or default_threads()
    zre, zim = np.zeros((npaths, n)), np.zeros((npaths, n))
    status, steps = np.zeros(npaths, np.int32), np.zeros(npaths, np.int32)
    tend = np.zeros(npaths)
    rc = lib().oracle_track(*T.args(), float(np.real(gamma)), float(np.imag(gamma)),
                            ctypes.byref(opts), int(path0), int(npaths), int(nthreads),
                            _d(zre), _d(zim), _i(status), _i(steps), _d(tend))
    if rc:
        raise ValueError("oracle_track: invalid arguments")
    return dict(z=zre + 1j * zim, status=status, steps=steps, tend=tend,
                path=np.arange(path0, path0 + npaths, dtype=np.int64))


def endgame(T: Terms, gamma: complex, paths, track_opts: TrackOpts | None = None,
            eg_opts: EgOpts | None = None, nthreads: int | None = None) -> dict:
    """Cauchy endgame for the listed paths: tracked to t = 1 - r0, then turns around t = 1
    (nphc_oracle.c, section "Cauchy endgame").  Returns the endpoint estimates z (path x n),
    status (EG_*), cycle numbers, the radius of the last turn and the distance between the
    last two estimates."""
    n = T.n
    paths = np.ascontiguousarray(paths, dtype=np.int64)
    cnt = paths.shape[0]
    track_opts = track_opts or default_track_opts()
    eg_opts = eg_opts or default_eg_opts()
    nthreads = nthreads or default_threads()
    zre, zim = np.zeros((cnt, n)), np.zeros((cnt, n))
    status, cycle = np.zeros(cnt, np.int32), np.zeros(cnt, np.int32)
    r_last, delta = np.zeros(cnt), np.zeros(cnt)
    rc = lib().oracle_endgame(*T.args(), float(np.real(gamma)), float(np.imag(gamma)),
                              ctypes.byref(track_opts), ctypes.byref(eg_opts),
                              paths.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cnt,
                              int(nthreads), _d(zre), _d(zim), _i(status), _i(cycle),
                              _d(r_last), _d(delta))
    if rc:
        raise ValueError("oracle_endgame: invalid arguments")
    return dict(z=zre + 1j * zim, status=status, cycle=cycle, r_last=r_last, delta=delta,
                path=paths)


def refine_certify(T: Terms, tr: dict, opts: CertOpts | None = None,
                   nthreads: int | None = None) -> dict:
    n = T.n
    opts = opts or default_cert_opts()
    nthreads = nthreads or default_threads()
    z = tr["z"]
    cnt = z.shape[0]
    zre, zim = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
    st = np.ascontiguousarray(tr["status"], dtype=np.int32)
    tend = np.ascontiguousarray(tr["tend"], dtype=np.float64)
    cls = np.zeros(cnt, np.int32)
    alpha, beta, gam, res, alpha_re = (np.zeros(cnt) for _ in range(5))
    rc = lib().oracle_refine_certify(*T.args(), ctypes.byref(opts), cnt, int(nthreads),
                                     _d(zre), _d(zim), _i(st), _d(tend), _i(cls), _d(alpha),
                                     _d(beta), _d(gam), _d(res), _d(alpha_re))
    if rc:
        raise ValueError("oracle_refine_certify: invalid arguments")
    return dict(z=zre + 1j * zim, cls=cls, alpha=alpha, beta=beta, gamma=gam, res=res,
                alpha_re=alpha_re)


def dedup(n: int, rc: dict) -> int:
    z = rc["z"]
    zre, zim = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
    beta = np.ascontiguousarray(rc["beta"])
    gam = np.ascontiguousarray(rc["gamma"])
    cls = rc["cls"]
    return int(lib().oracle_dedup(n, z.shape[0], _d(zre), _d(zim), _d(beta), _d(gam), _i(cls)))


def xy_classify(N: int, J: np.ndarray, c: np.ndarray, s: np.ndarray) -> dict:
    m = N - 1
    Jc = np.ascontiguousarray(J, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    theta, hess = np.zeros(m), np.zeros((m, m))
    idx = np.zeros(1, np.int32)
    en, mn, ld = np.zeros(1), np.zeros(1), np.zeros(1)
    lib().oracle_xy_classify(N, _d(Jc), _d(c), _d(s), _d(theta), _i(idx), _d(en), _d(mn), _d(ld),
                             _d(hess))
    return dict(theta=theta, index=int(idx[0]), energy=float(en[0]), min_abs_eig=float(mn[0]),
                log_abs_det=float(ld[0]), hessian=hess)


def xy_adjoint(N: int, J: np.ndarray, theta: np.ndarray, g_energy: float,
               g_theta: np.ndarray | None = None) -> np.ndarray:
    """dL/dJ_ij (N x N symmetric) of a loss L(V*, theta*) at the real SP theta* (N-1
    angles), given dL/dV and dL/dtheta (implicit function theorem, envelope for V)."""
    Jc = np.ascontiguousarray(J, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    g = None if g_theta is None else np.ascontiguousarray(g_theta, dtype=np.float64)
    dJ = np.zeros((N, N))
    if lib().oracle_xy_adjoint(N, _d(Jc), _d(th), float(g_energy), None if g is None else _d(g), _d(dJ)):
        raise ValueError("singular Hessian at the stationary point")
    return dJ


def solve_system(T: Terms, gamma: complex, track_opts=None, cert_opts=None, nthreads=None,
                 path0: int = 0, npaths: int | None = None) -> dict:
    """Track, refine, certify and deduplicate every path of the total-degree homotopy."""
    tr = track(T, gamma, path0, npaths, track_opts, nthreads)
    rc = refine_certify(T, tr, cert_opts, nthreads)
    ndup = dedup(T.n, rc)
    out = dict(tr)
    out.update(rc)
    out["n_duplicates"] = ndup
    return out


def solve_xy(N: int, sigma: float, gamma: complex, g: np.ndarray | None = None,
             eps: float = 0.1, track_opts=None, cert_opts=None, nthreads=None,
             path0: int = 0, npaths: int | None = None) -> dict:
    """The whole method for the power-law XY ring; real SPs are classified."""
    J = couplings(N, sigma, g, eps)
    T = xy_terms(N, J)
    out = solve_system(T, gamma, track_opts, cert_opts, nthreads, path0, npaths)
    m = N - 1
    real = np.nonzero(out["cls"] == C_REAL)[0]
    sps = []
    for i in real:
        z = out["z"][i]
        cl = xy_classify(N, J, z[:m].real, z[m:].real)
        cl["path"] = int(out["path"][i])
        cl["alpha"] = float(out["alpha"][i])
        cl["z"] = z
        sps.append(cl)
    out["J"] = J
    out["N"] = N
    out["sps"] = sps
    return out
