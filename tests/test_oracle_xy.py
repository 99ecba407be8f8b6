"""Pins for the oracle on the power-law XY ring (arXiv:1104.5497, section "A First
Application"): the paper's stationary-point counts, an independent brute force, closed-
form stationary points, structural identities and symmetries."""
import functools
import itertools
import os

import numpy as np
import pytest

import brute_force as B
import oracle as O
from oracle_cases import certified, load_counts, paper, real_thetas, xy
from paper_1104_5497_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
COUNTS = load_counts(os.path.join(GOLDEN, "paper_sp_counts.txt"))


def torus_dist(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b)))).max(axis=-1)


def contains(thetas, th, tol=1e-8):
    return len(thetas) > 0 and torus_dist(thetas, th).min() < tol


@pytest.mark.parametrize("N", [3, 5, 7])
def test_paper_counts(N):
    out = paper(N)
    assert len(out["sps"]) == COUNTS[N]
    assert out["n_duplicates"] == 0


@pytest.mark.slow
def test_paper_count_n9():
    out = paper(9)
    assert len(out["sps"]) == COUNTS[9]
    assert out["n_duplicates"] == 0


@pytest.mark.parametrize("N,sigma", [(3, 0.75), (4, 1.5), (5, 0.75), (5, 2.5)])
def test_brute_force_real_set(N, sigma):
    """Angle-grid Newton in theta (no homotopy) finds the same nonsingular real SPs,
    with the same Hessian index and energy."""
    out = xy(N, sigma, 11)
    J = B.ring_couplings(N, sigma)
    assert np.allclose(J, out["J"], rtol=1e-15, atol=0)
    th_b, idx_b, en_b, _ = B.real_stationary_points(N, J, grid=24 if N <= 4 else 14,
                                                     n_random=2000)
    th_o = real_thetas(out)
    assert len(th_o) == len(th_b)
    for th, ib, eb in zip(th_b, idx_b, en_b):
        k = torus_dist(th_o, th).argmin()
        assert torus_dist(th_o[k], th) < 1e-9
        assert out["sps"][k]["index"] == ib
        assert abs(out["sps"][k]["energy"] - eb) < 1e-10


@pytest.mark.parametrize("N,sigma", [(3, 0.75), (4, 1.5), (5, 0.75), (6, 1.5), (7, 0.75)])
def test_collinear_states(N, sigma):
    """Every theta in {0, pi}^(N-1) is stationary (all sines vanish); the oracle must
    certify exactly those whose Hessian is nonsingular, with V = sum J (1 - s_i s_j)."""
    out = xy(N, sigma, 11)
    J = out["J"]
    th_o = real_thetas(out)
    for bits in itertools.product([0, 1], repeat=N - 1):
        th = np.pi * np.array(bits, float)
        _, H = B.grad_hess(th[None], J)
        ev = np.linalg.eigvalsh(H[0])
        spins = np.append(np.cos(th), 1.0)
        V = 0.5 * (J * (1 - np.outer(spins, spins))).sum()
        if np.abs(ev).min() > 1e-9:
            assert contains(th_o, th)
            k = torus_dist(th_o, th).argmin()
            assert out["sps"][k]["index"] == (ev < 0).sum()
            assert abs(out["sps"][k]["energy"] - V) < 1e-10
        else:
            assert not contains(th_o, th, 1e-6)


def twisted_closed_form(N, sigma, n):
    """theta_k = 2 pi n k / N on a circulant ring: the Hessian is circulant, with
    eigenvalues lambda_q = sum_d J(d) cos(2 pi n d / N) (1 - cos(2 pi q d / N)); removing
    the pinned row and column drops only the q = 0 zero mode.  V = N/2 sum_d J(d)
    (1 - cos(2 pi n d / N))."""
    d = np.arange(1, N)
    Jd = np.minimum(d, N - d).astype(float) ** (-sigma)
    c = np.cos(2 * np.pi * n * d / N)
    lam = np.array([(Jd * c * (1 - np.cos(2 * np.pi * q * d / N))).sum() for q in range(1, N)])
    V = N / 2 * (Jd * (1 - c)).sum()
    return lam, V


@pytest.mark.parametrize("N,sigma", [(3, 0.75), (5, 0.75), (6, 1.5), (7, 0.75), (7, 2.5)])
def test_twisted_states(N, sigma):
    """Stationary-wave solutions theta_m = 2 pi m n / N (section 'A First Application')."""
    out = xy(N, sigma, 11)
    th_o = real_thetas(out)
    for n in range(N):
        lam, V = twisted_closed_form(N, sigma, n)
        th = np.angle(np.exp(2j * np.pi * n * np.arange(1, N) / N))
        if np.abs(lam).min() < 1e-9:
            continue
        assert contains(th_o, th)
        k = torus_dist(th_o, th).argmin()
        assert out["sps"][k]["index"] == (lam < 0).sum()
        assert abs(out["sps"][k]["energy"] - V) < 1e-10


@pytest.mark.parametrize("N,sigma", [(3, 0.75), (5, 0.75), (6, 1.5), (7, 0.75)])
def test_ferromagnetic_global_minimum(N, sigma):
    """The global minimum is all theta_i = 0 with V = 0 (section 'A First Application')."""
    out = xy(N, sigma, 11)
    en = np.array([s["energy"] for s in out["sps"]])
    k = en.argmin()
    assert abs(en[k]) < 1e-12
    assert np.abs(out["sps"][k]["theta"]).max() < 1e-12
    assert out["sps"][k]["index"] == 0
    assert (en[np.arange(len(en)) != k] > 1e-6).all()


@pytest.mark.parametrize("N,sigma", [(4, 1.5), (6, 1.5), (7, 0.75)])
def test_bezout_and_statuses(N, sigma):
    out = xy(N, sigma, 11)
    P = 4 ** (N - 1)
    assert len(out["status"]) == P
    assert (out["status"] != 0).all()
    assert certified(out).sum() <= P


@pytest.mark.parametrize("N,sigma", [(5, 0.75), (6, 1.5), (7, 0.75)])
def test_jacobian_hessian_determinant_identity(N, sigma):
    """At a real SP, in coordinates (theta, r) with c = r cos theta, s = r sin theta the
    Jacobian is [[H_theta, *], [0, 2 I]]; each pair d(c, s)/d(theta, r) has determinant
    -r = -1, so det DP = (-1)^(N-1) 2^(N-1) det H_theta.  Ties the term list to the
    classifier's Hessian."""
    out = xy(N, sigma, 11)
    T = O.xy_terms(N, out["J"])
    for s in out["sps"][:25]:
        _, D = T.eval_jac(s["z"].real)
        ratio = np.linalg.det(D) / ((-2) ** (N - 1) * np.linalg.det(s["hessian"]))
        assert abs(ratio - 1) < 1e-9
        # the classifier's log |det H| (sum of log |eigenvalue|) by the same identity
        ld = np.log(abs(np.linalg.det(D))) - (N - 1) * np.log(2.0)
        assert abs(ld - s["log_abs_det"]) < 1e-9 * max(1.0, abs(ld))


def test_d2_norm_closed_form():
    """||D^2 P / 2|| bound: each free pair contributes J_kj^2 to ||M_fk||_F^2 and each
    constraint c^2 + s^2 - 1 contributes 2."""
    for N, sigma in [(4, 1.5), (8, 0.75)]:
        J = B.ring_couplings(N, sigma)
        m = N - 1
        T = O.xy_terms(N, J)
        assert T.d2_norm() == pytest.approx(np.sqrt((J[:m, :m] ** 2).sum() + 2 * m), rel=1e-14)


@pytest.mark.parametrize("N,sigma", [(5, 0.75), (6, 1.5), (7, 0.75)])
def test_symmetries(N, sigma):
    """theta -> -theta, the ring reflection k -> N-k and re-pinned translations map the
    certified real set to itself, keeping energy and index; non-real certified
    solutions come in conjugate pairs (P has real coefficients)."""
    out = xy(N, sigma, 11)
    th = real_thetas(out)
    idx = np.array([s["index"] for s in out["sps"]])
    en = np.array([s["energy"] for s in out["sps"]])
    full = np.concatenate([th, np.zeros((len(th), 1))], axis=1)   # theta_N = 0 appended
    maps = [lambda f: -f, lambda f: f[:, [(N - 2 - k) % N for k in range(N - 1)] + [N - 1]]]
    for s in range(1, N):
        maps.append(lambda f, s=s: np.roll(f, -s, axis=1) - np.roll(f, -s, axis=1)[:, -1:])
    for mp in maps:
        img = np.angle(np.exp(1j * mp(full)[:, :N - 1]))
        for a in range(len(img)):
            k = torus_dist(th, img[a]).argmin()
            assert torus_dist(th[k], img[a]) < 1e-8
            assert idx[k] == idx[a] and abs(en[k] - en[a]) < 1e-10
    nr = out["z"][out["cls"] == O.C_NONREAL]
    for z in nr:
        assert np.linalg.norm(nr - z.conj(), axis=1).min() < 1e-9 * (1 + np.linalg.norm(z))


@pytest.mark.parametrize("N,sigma", [(5, 0.75), (6, 1.5)])
def test_gamma_independence(N, sigma):
    """For generic gamma every isolated solution is reached (section 'Numerical Polynomial
    Homotopy Continuation Method'): two gammas give the same certified set."""
    a = xy(N, sigma, 11)
    b = xy(N, sigma, 12)
    za = a["z"][certified(a)]
    zb = b["z"][certified(b)]
    assert len(za) == len(zb)
    for z in za:
        assert np.linalg.norm(zb - z, axis=1).min() < 1e-9 * (1 + np.linalg.norm(z))


@pytest.mark.parametrize("N,sigma", [(5, 0.75), (7, 0.75)])
def test_real_tolerance_stability(N, sigma):
    """The real count does not change below Delta_R ~ 1e-7 (same section), and the
    tolerance filter agrees with the alpha-theory real test."""
    out = xy(N, sigma, 11)
    cert = certified(out)
    im = np.abs(out["z"].imag).max(axis=1)
    counts = {tol: int((cert & (im <= tol)).sum()) for tol in (1e-6, 1e-7, 1e-8, 1e-10)}
    assert len(set(counts.values())) == 1
    assert counts[1e-7] == (out["cls"] == O.C_REAL).sum()
    assert (out["cls"] == O.C_UNDECIDED).sum() == 0


def test_disordered_couplings_are_symmetric_and_scaled():
    inst = I.disordered_batch(2, seed=3)[0]
    J = O.couplings(inst.N, inst.sigma, inst.g, inst.eps)
    J0 = B.ring_couplings(inst.N, inst.sigma, inst.g, inst.eps)
    assert np.allclose(J, J.T, rtol=0, atol=0) and np.allclose(J, J0, rtol=1e-15, atol=0)


@functools.lru_cache(maxsize=None)
def _brute_n5():
    return B.real_stationary_points(5, B.ring_couplings(5, 0.75), grid=14)[0]


@pytest.mark.parametrize("plant", ["pinned_sign", "drop_term", "transpose"])
def test_planted_mistake_is_caught(plant):
    """A plausible mistake in the polynomial system breaks agreement with the brute
    force (theta-space Newton on the true potential): the pins have teeth."""
    N, sigma = 5, 0.75
    J = O.couplings(N, sigma)
    T = O.xy_terms(N, J)
    if plant == "pinned_sign":        # s_k c_N entered with the wrong sign
        k = np.nonzero(T.vb == -1)[0][0]
        T.cre[k] = -T.cre[k]
    elif plant == "drop_term":        # one J s_j c_k term forgotten
        k = np.nonzero(T.cre < 0)[0][1]
        T.cre[k] = 0.0
    else:                             # s_k c_j written as s_j c_k in one term
        k = np.nonzero((T.vb >= 0) & (T.cre > 0) & (T.va != T.vb))[0][0]
        T.va[k], T.vb[k] = T.vb[k] + N - 1, T.va[k] - (N - 1)
    out = O.solve_system(T, I.paper_ring(N).gamma)
    m = N - 1
    zr = out["z"][out["cls"] == O.C_REAL].real
    th_o = np.angle(zr[:, :m] + 1j * zr[:, m:])
    th_b = _brute_n5()
    same = len(th_o) == len(th_b) and all(contains(th_o, t, 1e-8) for t in th_b)
    assert not same


def test_disordered_rings_share_one_finite_count():
    """The disordered N = 6 rings of the 64-ring batch workload: J_ij = d_ij^-sigma
    (1 + 0.1 g_ij) with random sigma and g are generic, and the number of isolated finite
    solutions of a square system is the same for every generic choice of its
    coefficients, so every ring certifies the same number (252, none singular), and two
    gammas give the same set on the ring with the largest solutions (norm 1.3e5).  A
    radius of 1e4 for paths to infinity certified 244 .. 252 on these rings."""
    rings = [r for r in I.disordered_batch(64, seed=3) if r.N == 6]
    assert len(rings) >= 8
    counts = set()
    for r in rings:
        out = O.solve_xy(r.N, r.sigma, r.gamma, g=r.g, eps=r.eps)
        assert (out["cls"] == O.C_SINGULAR).sum() == 0
        counts.add(int(certified(out).sum()))
    assert counts == {252}
    far = I.disordered_batch(64, seed=3)[24]
    zs = []
    for gam in (far.gamma, np.exp(2.1j)):
        out = O.solve_xy(far.N, far.sigma, gam, g=far.g, eps=far.eps)
        zs.append(out["z"][certified(out)])
    assert np.abs(zs[0]).max() > 1e5
    assert len(zs[0]) == len(zs[1])
    for z in zs[0]:
        assert np.linalg.norm(zs[1] - z, axis=1).min() < 1e-9 * (1 + np.linalg.norm(z))
