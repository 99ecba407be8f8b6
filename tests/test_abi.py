"""The C ABI without a GPU: the library builds, loads and exports every function that
include/nphc.h declares; host-side argument checks and the couplings builder."""
import os
import re

import numpy as np
import pytest

import brute_force as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def N_():
    from paper_1104_5497_gb300 import build
    build.build()
    import paper_1104_5497_gb300.nphc as nphc
    return nphc


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nphc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nphc_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(N_):
    names = declared_functions()
    assert len(names) >= 20
    L = N_.lib()
    for name in names:
        assert hasattr(L, name), name


def test_options_defaults(N_):
    o = N_.options_default()
    assert o.precision == N_.PREC_MIXED
    assert o.tol_sol == 1e-10 and o.tol_real == 1e-7
    assert abs(o.gamma_re ** 2 + o.gamma_im ** 2 - 1) < 1e-15


@pytest.mark.parametrize("N,sigma", [(3, 0.75), (8, 1.5), (13, 1.0)])
def test_couplings_builder(N_, N, sigma):
    assert np.array_equal(N_.xy_couplings(N, sigma), B.ring_couplings(N, sigma))


def test_disordered_couplings_builder(N_):
    rng = np.random.default_rng(0)
    g = rng.standard_normal((7, 7))
    g = np.triu(g, 1) + np.triu(g, 1).T
    J = N_.xy_couplings(7, 1.2, g, 0.1)
    assert np.allclose(J, B.ring_couplings(7, 1.2, g, 0.1), rtol=1e-15, atol=0)


@pytest.mark.parametrize("disorder", [False, True])
def test_couplings_vjp_is_the_sigma_derivative(N_, disorder):
    """nphc_xy_couplings_vjp against central differences of nphc_xy_couplings in sigma,
    for a random dL/dJ (diagonal ignored), with and without per-pair disorder."""
    rng = np.random.default_rng(3)
    N, sigma = 9, 1.3
    g = None
    if disorder:
        g = rng.standard_normal((N, N))
        g = np.triu(g, 1) + np.triu(g, 1).T
    w = rng.standard_normal((N, N))
    h = 1e-6
    fd = float(((N_.xy_couplings(N, sigma + h, g, 0.1) - N_.xy_couplings(N, sigma - h, g, 0.1)) * w).sum()) / (2 * h)
    got = N_.xy_couplings_vjp(N, sigma, w, g, 0.1)
    assert abs(got - fd) < 1e-8 * (1 + abs(fd))
    w0 = w.copy()
    np.fill_diagonal(w0, 1e3)
    assert N_.xy_couplings_vjp(N, sigma, w0, g, 0.1) == N_.xy_couplings_vjp(N, sigma, w - np.diag(np.diag(w)), g, 0.1)


def test_invalid_arguments_are_reported(N_):
    for N in (2, 14):
        with pytest.raises(N_.NphcError) as ei:
            N_.System(N, 1.0)
        assert ei.value.status == 1
    J = N_.xy_couplings(5, 1.0)
    J[0, 1] += 1e-3
    with pytest.raises(N_.NphcError):
        N_.System(5, 1.0, J)
    J = N_.xy_couplings(5, 1.0)
    J[2, 3] = J[3, 2] = np.nan
    with pytest.raises(N_.NphcError):
        N_.System(5, 1.0, J)
    g = np.ones((5, 5))
    g[0, 1] = 2.0
    with pytest.raises(N_.NphcError):
        N_.xy_couplings(5, 1.0, g, 0.1)


@pytest.mark.parametrize("N", [3, 10, 13])
def test_system_dimensions(N_, N):
    s = N_.System(N, 1.0)
    assert (s.N, s.n, s.npaths) == (N, 2 * (N - 1), 4 ** (N - 1))
    assert np.array_equal(s.couplings(), B.ring_couplings(N, 1.0))
    assert s.workspace_size(1000) < s.workspace_size(100000)


def test_quadratic_system_argument_checks(N_):
    """nphc_system_create_quadratic validates the term list before touching the device."""
    ok = dict(eq=[0, 0], va=[0, -1], vb=[0, -1], coef=[1.0, -5.0])
    bad = [
        (0, ok), (N_.QUAD_MAX_N + 1, ok),
        (1, dict(ok, eq=[0, 1])),                      # equation index out of range
        (1, dict(ok, va=[0, -2])),                     # variable index out of range
        (1, dict(ok, vb=[1, -1])),
        (1, dict(ok, coef=[1.0, float("nan")])),
    ]
    for n, t in bad:
        with pytest.raises(N_.NphcError) as ei:
            N_.System.quadratic(n, t["eq"], t["va"], t["vb"], t["coef"])
        assert ei.value.status == 1


def test_endgame_argument_checks(N_):
    """nphc_endgame rejects bad endgame options and missing outputs before any CUDA call
    (the endpoint pointers below are never dereferenced)."""
    import ctypes
    s = N_.System(5, 1.0)
    ep = N_.nphc_endpoints()
    ep.count = 4
    for f in ("path", "z_re", "z_im", "t", "h", "status", "steps", "solves", "newton"):
        setattr(ep, f, 16)
    L = N_.lib()
    dummy = ctypes.c_void_p(16)
    bad = [dict(eg_r0=1.5), dict(eg_r0=0.0), dict(eg_ratio=1.0), dict(eg_radii=0),
           dict(eg_samples=1), dict(eg_samples=5000), dict(eg_max_cycle=0),
           dict(eg_tol_close=0.0), dict(eg_tol_conv=-1.0), dict(eg_h_min=0.0),
           dict(eg_max_attempts=0)]
    for kw in bad:
        o = N_.options_default(**kw)
        rc = L.nphc_endgame(s.handle, ctypes.byref(o), ctypes.byref(ep), None, None, dummy, dummy,
                            dummy, 1 << 40, None)
        assert rc == 1, kw
        assert b"endgame options" in L.nphc_last_error()
    o = N_.options_default()
    rc = L.nphc_endgame(s.handle, ctypes.byref(o), ctypes.byref(ep), None, None, None, dummy,
                        dummy, 1 << 40, None)
    assert rc == 1 and b"cycle" in L.nphc_last_error()
    d = N_.options_default()
    assert (d.endgame, d.eg_r0, d.eg_ratio, d.eg_radii, d.eg_samples, d.eg_max_cycle) == \
        (0, 1 / 16, 0.25, 8, 16, 8)


def test_launch_options_are_checked(N_):
    """Negative launch shapes are rejected before any CUDA call."""
    import ctypes
    s = N_.System(5, 1.0)
    ep = N_.nphc_endpoints()
    ep.count = 4
    for f in ("path", "z_re", "z_im", "t", "h", "status", "steps", "solves", "newton"):
        setattr(ep, f, 16)
    L = N_.lib()
    for kw in (dict(blocks_per_sm=-1), dict(list_blocks_per_sm=-2), dict(block_size=-1)):
        o = N_.options_default(**kw)
        rc = L.nphc_track(s.handle, ctypes.byref(o), N_.PREC_MIXED, ctypes.byref(ep), None, None, 0,
                          ctypes.c_void_p(16), 1 << 40, None)
        assert rc == 1 and b"launch options" in L.nphc_last_error(), kw
    assert N_.options_default().list_blocks_per_sm == 0
