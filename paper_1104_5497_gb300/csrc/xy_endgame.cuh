// xy_endgame.cuh -- FP64 work at t = 1 on the endpoints of the XY ring:
//   refinement: Newton's method on P to machine precision (section "Numerical Polynomial
//     Homotopy Continuation Method": refinement "up to the machine precision"), with P
//     evaluated by exact products and double-double sums (xy_eval_p_acc);
//   the solution tolerance Delta_sol on ||P(z)||_inf;
//   alpha-theory certification (the alphaCertified step of the same section):
//     beta = ||DP^-1 P||_2, gamma <= ||DP^-1||_F ||D^2 P / 2|| (P is quadratic, so
//     D^k P = 0 for k >= 3 and Smale's gamma is ||DP^-1 D^2P/2|| exactly), certified when
//     alpha = beta gamma < (13 - 3 sqrt 17) / 4; real when the test passes at Re z (a real
//     point of a real system: Newton's iterates stay real), non-real when
//     ||z - conj z|| > 2 (beta(z) + beta(conj z)), i.e. ||Im z|| > 2 beta;
//   classification of real stationary points (introduction and section "A First
//     Application"): theta_k = atan2(s_k, c_k) in (-pi, pi], the Hessian of
//     V = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)) in theta_1..theta_M, its number of
//     negative eigenvalues (cyclic Jacobi), and V.
//
// The linear solves reuse the structure of xy_solve.cuh at t = 1 (a unitary frame per
// constraint row, an M x M Schur system factored once by Householder QR) but keep the
// factorisation in local memory so that it can be applied to many right-hand sides:
// ||DP^-1||_F^2 = sum_i ||DP^-1 e_i||^2 needs 2M of them.
#pragma once

#include "nphc_internal.cuh"

template <int M>
struct Fac64 {
    cx<double> A[M][M];   // R above the diagonal, Householder vectors below
    cx<double> tauc[M];   // conj(tau) of each reflector
    double dg[M];         // real diagonal of R
    cx<double> ah[M], bh[M];
    double iv[M];
    cx<double> Ad[M], Bd[M];   // diagonal Jacobian entries of the gradient rows
    cx<double> x[M], y[M];
    bool ok;
};

// P(z) (t = 1): gradient rows f_k and constraint rows g_k.
template <int M>
__device__ void xy_eval_p(const double *__restrict__ J, const cx<double> (&x)[M],
                          const cx<double> (&y)[M], cx<double> (&f)[M], cx<double> (&g)[M]) {
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        cx<double> u = cx<double>{J[k * NPHC_JSTRIDE + M], 0.0}, w = cx<double>{0.0, 0.0};
        for (int l = 0; l < M; l++) {
            if (l == k) continue;
            const double Jl = J[k * NPHC_JSTRIDE + l];
            u.re += Jl * x[l].re;
            u.im += Jl * x[l].im;
            w.re += Jl * y[l].re;
            w.im += Jl * y[l].im;
        }
        f[k] = csub(cmul(y[k], u), cmul(x[k], w));
        const cx<double> x2 = cmul(x[k], x[k]), y2 = cmul(y[k], y[k]);
        g[k] = cx<double>{x2.re + y2.re - 1.0, x2.im + y2.im};
    }
}

// P(z) with exact products and double-double sums, rounded once: at ||z|| >> 1 the
// terms of P are ~||z||^2 and a plain double sum is dominated by rounding, which would
// limit the refinement and inflate beta (hence alpha) of large-norm solutions.
struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_two_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    return dd{p, __fma_rn(a, b, -p)};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
    const double s = __dadd_rn(a.hi, b.hi);
    const double bb = __dsub_rn(s, a.hi);
    const double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bb)), __dsub_rn(b.hi, bb));
    const double lo = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
    const double hi = __dadd_rn(s, lo);
    return dd{hi, __dsub_rn(lo, __dsub_rn(hi, s))};
}

// a * b with a double-double, b double
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    const dd p = dd_two_prod(a.hi, b);
    const double lo = __fma_rn(a.lo, b, p.lo);
    const double hi = __dadd_rn(p.hi, lo);
    return dd{hi, __dsub_rn(lo, __dsub_rn(hi, p.hi))};
}

__device__ __forceinline__ double dd_val(dd a) { return __dadd_rn(a.hi, a.lo); }

template <int M>
__device__ void xy_eval_p_acc(const double *__restrict__ J, const cx<double> (&x)[M],
                              const cx<double> (&y)[M], cx<double> (&f)[M], cx<double> (&g)[M]) {
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const double *Jk = J + k * NPHC_JSTRIDE;
        dd ur = {Jk[M], 0.0}, ui = {0.0, 0.0}, wr = {0.0, 0.0}, wi = {0.0, 0.0};
        for (int l = 0; l < M; l++) {   // J_kk = 0 adds exact zeros
            ur = dd_add(ur, dd_two_prod(Jk[l], x[l].re));
            ui = dd_add(ui, dd_two_prod(Jk[l], x[l].im));
            wr = dd_add(wr, dd_two_prod(Jk[l], y[l].re));
            wi = dd_add(wi, dd_two_prod(Jk[l], y[l].im));
        }
        // f = y u - x w
        dd fr = dd_add(dd_add(dd_mul_d(ur, y[k].re), dd_mul_d(ui, -y[k].im)),
                       dd_add(dd_mul_d(wr, -x[k].re), dd_mul_d(wi, x[k].im)));
        dd fi = dd_add(dd_add(dd_mul_d(ui, y[k].re), dd_mul_d(ur, y[k].im)),
                       dd_add(dd_mul_d(wi, -x[k].re), dd_mul_d(wr, -x[k].im)));
        // g = c^2 + s^2 - 1
        dd gr = dd_add(dd_add(dd_two_prod(x[k].re, x[k].re), dd_two_prod(-x[k].im, x[k].im)),
                       dd_add(dd_two_prod(y[k].re, y[k].re), dd_two_prod(-y[k].im, y[k].im)));
        gr = dd_add(gr, dd{-1.0, 0.0});
        dd gi = dd_add(dd_two_prod(2.0 * x[k].re, x[k].im), dd_two_prod(2.0 * y[k].re, y[k].im));
        f[k] = cx<double>{dd_val(fr), dd_val(fi)};
        g[k] = cx<double>{dd_val(gr), dd_val(gi)};
    }
}

// Factor DP(z) (t = 1).
template <int M>
__device__ void fac_build(Fac64<M> &F, const double *__restrict__ J) {
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        cx<double> u = cx<double>{J[j * NPHC_JSTRIDE + M], 0.0}, w = cx<double>{0.0, 0.0};
        for (int l = 0; l < M; l++) {
            if (l == j) continue;
            const double Jl = J[j * NPHC_JSTRIDE + l];
            u.re += Jl * F.x[l].re;
            u.im += Jl * F.x[l].im;
            w.re += Jl * F.y[l].re;
            w.im += Jl * F.y[l].im;
        }
        F.Ad[j] = cx<double>{-w.re, -w.im};   // d f_j / d c_j
        F.Bd[j] = u;                          // d f_j / d s_j
        const cx<double> a = cscale(2.0, F.x[j]), b = cscale(2.0, F.y[j]);
        const double iv = rsqrt(cabs2(a) + cabs2(b));
        F.iv[j] = iv;
        F.ah[j] = cscale(iv, a);
        F.bh[j] = cscale(iv, b);
    }
#pragma unroll 1
    for (int j = 0; j < M; j++)
        for (int k = 0; k < M; k++) {
            if (k == j)
                F.A[k][j] = csub(cmul(F.Ad[j], F.bh[j]), cmul(F.Bd[j], F.ah[j]));
            else
                F.A[k][j] = cscale(J[k * NPHC_JSTRIDE + j],
                                   cadd(cmul(F.y[k], F.bh[j]), cmul(F.x[k], F.ah[j])));
        }
    F.ok = true;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const cx<double> al = F.A[k][k];
        double xn2 = 0.0;
        for (int i = k + 1; i < M; i++) xn2 += cabs2(F.A[i][k]);
        const double an = sqrt(cabs2(al) + xn2);
        F.ok = F.ok && an > 0.0;
        const double beta = al.re >= 0.0 ? -an : an;
        F.tauc[k] = cx<double>{(beta - al.re) / beta, al.im / beta};
        const cx<double> sc = crecip(cx<double>{al.re - beta, al.im});
        for (int i = k + 1; i < M; i++) F.A[i][k] = cmul(F.A[i][k], sc);
        F.dg[k] = beta;
        for (int c = k + 1; c < M; c++) {
            cx<double> wv = F.A[k][c];
            for (int i = k + 1; i < M; i++) wv = cadd(wv, cmulc(F.A[i][k], F.A[i][c]));
            wv = cmul(F.tauc[k], wv);
            F.A[k][c] = csub(F.A[k][c], wv);
            for (int i = k + 1; i < M; i++) F.A[i][c] = csub(F.A[i][c], cmul(F.A[i][k], wv));
        }
    }
}

// d = DP^-1 r for r = (rf, rg); returns ||d||_2^2.
template <int M>
__device__ double fac_apply(const Fac64<M> &F, const double *__restrict__ J,
                            const cx<double> (&rf)[M], const cx<double> (&rg)[M],
                            cx<double> (&dx)[M], cx<double> (&dy)[M]) {
    cx<double> q[M], b[M];
#pragma unroll 1
    for (int j = 0; j < M; j++) q[j] = cscale(F.iv[j], rg[j]);
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        cx<double> acc = rf[k];
        for (int j = 0; j < M; j++) {
            const cx<double> px = cmulc(F.ah[j], q[j]), py = cmulc(F.bh[j], q[j]);
            if (k == j)
                acc = csub(acc, cadd(cmul(F.Ad[j], px), cmul(F.Bd[j], py)));
            else
                acc = csub(acc, cscale(J[k * NPHC_JSTRIDE + j],
                                       csub(cmul(F.y[k], px), cmul(F.x[k], py))));
        }
        b[k] = acc;
    }
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        cx<double> wv = b[k];
        for (int i = k + 1; i < M; i++) wv = cadd(wv, cmulc(F.A[i][k], b[i]));
        wv = cmul(F.tauc[k], wv);
        b[k] = csub(b[k], wv);
        for (int i = k + 1; i < M; i++) b[i] = csub(b[i], cmul(F.A[i][k], wv));
    }
#pragma unroll 1
    for (int k = M - 1; k >= 0; k--) {
        cx<double> acc = b[k];
        for (int c = k + 1; c < M; c++) acc = csub(acc, cmul(F.A[k][c], b[c]));
        b[k] = cscale(1.0 / F.dg[k], acc);
    }
    double n2 = 0.0;
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        dx[j] = cadd(cmulc(F.ah[j], q[j]), cmul(F.bh[j], b[j]));
        dy[j] = csub(cmulc(F.bh[j], q[j]), cmul(F.ah[j], b[j]));
        n2 += cabs2(dx[j]) + cabs2(dy[j]);
    }
    return n2;
}

// beta = ||DP^-1 P||, ||DP^-1||_F and ||P||_inf at (x, y).  Returns false if singular.
template <int M>
__device__ bool xy_beta_invnorm(Fac64<M> &F, const double *__restrict__ J, double &beta,
                                double &invF, double &res) {
    cx<double> f[M], g[M], dx[M], dy[M];
    xy_eval_p_acc<M>(J, F.x, F.y, f, g);
    res = 0.0;
    for (int k = 0; k < M; k++) {
        res = fmax(res, sqrt(cabs2(f[k])));
        res = fmax(res, sqrt(cabs2(g[k])));
        f[k] = cx<double>{-f[k].re, -f[k].im};
        g[k] = cx<double>{-g[k].re, -g[k].im};
    }
    fac_build<M>(F, J);
    if (!F.ok) return false;
    beta = sqrt(fac_apply<M>(F, J, f, g, dx, dy));
    double s = 0.0;
#pragma unroll 1
    for (int i = 0; i < 2 * M; i++) {
        for (int k = 0; k < M; k++) {
            f[k] = cx<double>{i == k ? 1.0 : 0.0, 0.0};
            g[k] = cx<double>{i == M + k ? 1.0 : 0.0, 0.0};
        }
        s += fac_apply<M>(F, J, f, g, dx, dy);
    }
    invF = sqrt(s);
    return isfinite(beta) && isfinite(invF);
}

// shortcut = 1: entries handed off by the FP32 pass close to t = 1 are refined at t = 1
// directly (Newton on P from the hand-off point: for a path to a nonsingular solution xi,
// z(t) = xi + (1 - t) z'(1) + ..., so the point is already in xi's Newton basin).  The
// first Newton correction must stay below SHORTCUT_TRUST (1 + ||z||); an entry that
// certifies becomes NPHC_PATH_REACHED, any other entry is left untouched.
#define SHORTCUT_TRUST 1e-2

template <int M>
__global__ void __launch_bounds__(128)
    xy_refine_certify_kernel(const __grid_constant__ XYSys S, double tol_sol, double refine_eps,
                             int refine_iters, const EPView ep, const WorkList wl, int shortcut) {
    const int64_t total = worklist_size(wl, ep.count);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int64_t e = worklist_entry(wl, i);
    const int64_t cnt = ep.count;
    const int st = ep.status[e];
    const bool sc = shortcut && st == NPHC_PATH_HANDOFF;
    if (!sc) {
        ep.alpha[e] = INFINITY;
        ep.beta[e] = INFINITY;
        ep.gamma[e] = INFINITY;
        ep.resid[e] = INFINITY;
        if (st == NPHC_PATH_DIVERGED) {
            ep.cls[e] = NPHC_END_NONE;
            return;
        }
        if (st != NPHC_PATH_REACHED) {
            ep.cls[e] = NPHC_END_FAILED;
            return;
        }
    }
    const double *J = S.Jd;
    const double alpha0 = (13.0 - 3.0 * sqrt(17.0)) / 4.0;
    Fac64<M> F;
    for (int k = 0; k < M; k++) {
        F.x[k] = cx<double>{ep.z_re[k * cnt + e], ep.z_im[k * cnt + e]};
        F.y[k] = cx<double>{ep.z_re[(M + k) * cnt + e], ep.z_im[(M + k) * cnt + e]};
    }
    int cls = NPHC_END_SINGULAR;
    bool finite = true;
    // Newton refinement on P
    for (int it = 0; it < refine_iters; it++) {
        cx<double> f[M], g[M], dx[M], dy[M];
        xy_eval_p_acc<M>(J, F.x, F.y, f, g);
        for (int k = 0; k < M; k++) {
            f[k] = cx<double>{-f[k].re, -f[k].im};
            g[k] = cx<double>{-g[k].re, -g[k].im};
        }
        fac_build<M>(F, J);
        if (!F.ok) break;
        const double dn = sqrt(fac_apply<M>(F, J, f, g, dx, dy));
        if (sc && it == 0) {
            double z0 = 0.0;
            for (int k = 0; k < M; k++) z0 += cabs2(F.x[k]) + cabs2(F.y[k]);
            if (!(dn <= SHORTCUT_TRUST * (1.0 + sqrt(z0)))) return;   // not in a basin: untouched
        }
        double zn = 0.0;
        for (int k = 0; k < M; k++) {
            F.x[k] = cadd(F.x[k], dx[k]);
            F.y[k] = cadd(F.y[k], dy[k]);
            zn += cabs2(F.x[k]) + cabs2(F.y[k]);
        }
        if (!isfinite(dn) || !isfinite(zn)) {
            finite = false;
            break;
        }
        if (dn <= refine_eps * (1.0 + sqrt(zn))) break;
    }
    double beta = INFINITY, invF = INFINITY, res = INFINITY;
    if (finite && xy_beta_invnorm<M>(F, J, beta, invF, res)) {
        const double gam = invF * S.d2norm, alpha = beta * gam;
        ep.alpha[e] = alpha;
        ep.beta[e] = beta;
        ep.gamma[e] = gam;
        ep.resid[e] = res;
        // Delta_sol relative to the size of the (quadratic) terms: max(1, ||z||_inf^2)
        double zi = 0.0;
        for (int k = 0; k < M; k++) zi = fmax(zi, fmax(sqrt(cabs2(F.x[k])), sqrt(cabs2(F.y[k]))));
        if (res <= tol_sol * fmax(1.0, zi * zi) && alpha < alpha0) {
            double im2 = 0.0;
            for (int k = 0; k < M; k++) im2 += F.x[k].im * F.x[k].im + F.y[k].im * F.y[k].im;
            if (sqrt(im2) > 2.0 * beta) {
                cls = NPHC_END_NONREAL;
            } else {
                // real test at Re z
                Fac64<M> G;
                for (int k = 0; k < M; k++) {
                    G.x[k] = cx<double>{F.x[k].re, 0.0};
                    G.y[k] = cx<double>{F.y[k].re, 0.0};
                }
                double br, ir, rr;
                if (xy_beta_invnorm<M>(G, J, br, ir, rr) && br * ir * S.d2norm < alpha0)
                    cls = NPHC_END_REAL;
                else
                    cls = NPHC_END_UNDECIDED;
            }
        }
    } else if (finite) {
        ep.resid[e] = res;
    }
    if (sc) {
        if (cls != NPHC_END_REAL && cls != NPHC_END_NONREAL && cls != NPHC_END_UNDECIDED) return;
        ep.status[e] = NPHC_PATH_REACHED;
        ep.t[e] = 1.0;
    }
    for (int k = 0; k < M; k++) {
        ep.z_re[k * cnt + e] = F.x[k].re;
        ep.z_im[k * cnt + e] = F.x[k].im;
        ep.z_re[(M + k) * cnt + e] = F.y[k].re;
        ep.z_im[(M + k) * cnt + e] = F.y[k].im;
    }
    ep.cls[e] = cls;
}

template <int M>
__global__ void __launch_bounds__(128)
    xy_classify_kernel(const __grid_constant__ XYSys S, const EPView ep, double *theta,
                       int32_t *index, double *energy, double *min_eig) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = ep.count;
    if (e >= cnt) return;
    if (ep.cls[e] != NPHC_END_REAL) {
        index[e] = -1;
        energy[e] = 0.0;
        if (min_eig) min_eig[e] = 0.0;
        for (int k = 0; k < M; k++) theta[k * cnt + e] = 0.0;
        return;
    }
    const double *J = S.Jd;
    constexpr int N = M + 1;
    double c[N], s[N];
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const double x = ep.z_re[k * cnt + e], y = ep.z_re[(M + k) * cnt + e];
        double a = atan2(y, x);
        if (a <= -M_PI) a = M_PI;
        sincos(a, &s[k], &c[k]);
        theta[k * cnt + e] = a;
    }
    c[M] = 1.0;   // theta_N = 0
    s[M] = 0.0;
    // V = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)), cos(a - b) = c_a c_b + s_a s_b
    double V = 0.0;
#pragma unroll 1
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) V += J[i * NPHC_JSTRIDE + j] * (1.0 - (c[i] * c[j] + s[i] * s[j]));
    // Hessian in theta_1..theta_M (row-major, flat)
    double H[M * M];
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        double d = 0.0;
        for (int j = 0; j < N; j++)
            if (j != k) d += J[k * NPHC_JSTRIDE + j] * (c[k] * c[j] + s[k] * s[j]);
        for (int l = 0; l < M; l++)
            H[k * M + l] = (k == l) ? d : -J[k * NPHC_JSTRIDE + l] * (c[k] * c[l] + s[k] * s[l]);
    }
    // cyclic Jacobi rotations until the off-diagonal part is negligible
#pragma unroll 1
    for (int sweep = 0; sweep < 64; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < M * M; i++) {
            tot += H[i] * H[i];
            if (i / M != i % M) off += H[i] * H[i];
        }
        if (off <= 1e-30 * tot) break;
#pragma unroll 1
        for (int p = 0; p < M - 1; p++)
#pragma unroll 1
            for (int q = p + 1; q < M; q++) {
                const double apq = H[p * M + q];
                if (apq == 0.0) continue;
                const double tq = (H[q * M + q] - H[p * M + p]) / (2.0 * apq);
                const double tn = (tq >= 0.0 ? 1.0 : -1.0) / (fabs(tq) + sqrt(tq * tq + 1.0));
                const double cs = 1.0 / sqrt(tn * tn + 1.0), sn = tn * cs;
#pragma unroll 1
                for (int k = 0; k < M; k++) {   // columns p and q
                    const double akp = H[k * M + p], akq = H[k * M + q];
                    H[k * M + p] = cs * akp - sn * akq;
                    H[k * M + q] = sn * akp + cs * akq;
                }
#pragma unroll 1
                for (int k = 0; k < M; k++) {   // rows p and q
                    const double apk = H[p * M + k], aqk = H[q * M + k];
                    H[p * M + k] = cs * apk - sn * aqk;
                    H[q * M + k] = sn * apk + cs * aqk;
                }
            }
    }
    int neg = 0;
    double mn = INFINITY;
    for (int k = 0; k < M; k++) {
        const double w = H[k * M + k];
        if (w < 0.0) neg++;
        mn = fmin(mn, fabs(w));
    }
    index[e] = neg;
    energy[e] = V;
    if (min_eig) min_eig[e] = mn;
}
