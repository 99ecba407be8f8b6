// xy_solve.cuh -- the linear algebra at the heart of every predictor and corrector
// step for the XY ring: solving H_z(z,t) d = r for the homotopy
//   H(z,t) = gamma (1-t) Q(z) + t P(z),  Q_i = z_i^2 - 1,
// with P the stationary equations of Eq. (alg_dec_XY_model_poly):
//   f_k = s_k u_k - c_k w_k,  u_k = sum_{j != k} J_kj c_j,  w_k = sum_{j != k} J_kj s_j,
//   g_k = c_k^2 + s_k^2 - 1,  (c_N, s_N) = (1, 0) pinned,
// unknowns z = (c_1..c_M, s_1..s_M), M = N-1 (called x and y below).
//
// Structure used: the constraint row of site k touches only (x_k, y_k):
//   a_k dx_k + b_k dy_k = r_gk,  a_k = 2 t x_k,  b_k = 2 (t + gamma (1-t)) y_k.
// A unitary change of variables per site, (dx_k, dy_k) = conj(a^, b^) q_k + (b^, -a^) s_k
// with (a^, b^) = (a_k, b_k) / |(a_k, b_k)|, turns that row into q_k = r_gk / |(a_k, b_k)|
// and leaves an M x M complex system for s in the gradient rows:
//   S_kj = A_kj b^_j - B_kj a^_j,   rhs_k = r_fk - sum_j (A_kj conj(a^_j) + B_kj conj(b^_j)) q_j,
// where A = d(f rows)/dx and B = d(f rows)/dy of H.  S is solved by Householder QR
// (unitary, so no pivot search and no data-dependent indexing: everything stays in
// registers of one thread).  Cost ~ (8/3) M^3 + O(M^2 + M N) instead of (8/3) (2M)^3.
#pragma once

#include "nphc_internal.cuh"

// One thread's vector of 2M complex unknowns in shared memory, interleaved across the
// threads of the block (component e of thread tid at [e * BLOCK + tid]): conflict-free.
template <class R, int BLOCK>
struct TVec {
    R *p;
    __device__ __forceinline__ cx<R> get(int i) const { return cx<R>{p[(2 * i) * BLOCK], p[(2 * i + 1) * BLOCK]}; }
    __device__ __forceinline__ void set(int i, cx<R> v) const {
        p[(2 * i) * BLOCK] = v.re;
        p[(2 * i + 1) * BLOCK] = v.im;
    }
};

__device__ __forceinline__ void compiler_fence() { asm volatile("" ::: "memory"); }

// -H_t(z) for gradient row k and constraint row k, H_t = P - gamma Q.
template <int M, class R>
__device__ __forceinline__ void xy_minus_ht(const R *__restrict__ J, const cx<R> (&x)[M],
                                            const cx<R> (&y)[M], int k, cx<R> gam, cx<R> &u,
                                            cx<R> &w, cx<R> &rf, cx<R> &rg) {
    u = cx<R>{J[k * NPHC_JSTRIDE + M], R(0)};
    w = cx<R>{R(0), R(0)};
#pragma unroll
    for (int l = 0; l < M; l++) {
        if (l == k) continue;
        const R Jl = J[k * NPHC_JSTRIDE + l];
        u.re += Jl * x[l].re;
        u.im += Jl * x[l].im;
        w.re += Jl * y[l].re;
        w.im += Jl * y[l].im;
    }
    const cx<R> f = csub(cmul(y[k], u), cmul(x[k], w));
    const cx<R> x2 = cmul(x[k], x[k]), y2 = cmul(y[k], y[k]);
    const cx<R> qx = cx<R>{x2.re - R(1), x2.im}, qy = cx<R>{y2.re - R(1), y2.im};
    const cx<R> g = cx<R>{x2.re + y2.re - R(1), x2.im + y2.im};
    rf = csub(cmul(gam, qx), f);
    rg = csub(cmul(gam, qy), g);
}

// Solve H_z(z, te) d = r for NR right-hand sides.
//   NR == 1: r = -H_t (predictor: d = dz/dt), written to out1.
//   NR == 2: r1 = the residual vector in `res` (corrector: -H), written to out1;
//            r2 = -H_t, written to out2.
// Outputs are written only when wr.  Returns false when the system is singular or the
// result is not finite.
template <int M, class R, int NR, int BLOCK>
__device__ __forceinline__ bool xy_solve(const R *__restrict__ J, const TVec<R, BLOCK> &pt,
                                         double te, cx<R> gam, const TVec<R, BLOCK> &res,
                                         const TVec<R, BLOCK> &out1, const TVec<R, BLOCK> &out2,
                                         bool wr) {
    const R s = (R)te;
    const R omt = (R)(1.0 - te);
    const cx<R> gomt = cscale(omt, gam);
    const cx<R> sg = cx<R>{s + gomt.re, gomt.im};   // t + gamma (1 - t)

    cx<R> x[M], y[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        x[k] = pt.get(k);
        y[k] = pt.get(M + k);
    }

    cx<R> A[M][M];
    cx<R> b[NR][M];
#pragma unroll
    for (int r = 0; r < NR; r++)
#pragma unroll
        for (int k = 0; k < M; k++) b[r][k] = cx<R>{R(0), R(0)};

    // ---- build the Schur system column by column
#pragma unroll
    for (int j = 0; j < M; j++) {
        cx<R> u, w, htf, htg;
        xy_minus_ht<M, R>(J, x, y, j, gam, u, w, htf, htg);
        cx<R> rf[NR], rg[NR];
        if constexpr (NR == 1) {
            rf[0] = htf;
            rg[0] = htg;
        } else {
            rf[0] = res.get(j);
            rg[0] = res.get(M + j);
            rf[1] = htf;
            rg[1] = htg;
        }
        // diagonal entries of the gradient rows
        const cx<R> Ajj = cx<R>{-s * w.re + R(2) * (gomt.re * x[j].re - gomt.im * x[j].im),
                                -s * w.im + R(2) * (gomt.re * x[j].im + gomt.im * x[j].re)};
        const cx<R> Bjj = cscale(s, u);
        // frame of constraint row j
        const cx<R> a = cscale(R(2) * s, x[j]);
        const cx<R> bb = cscale(R(2), cmul(sg, y[j]));
        const R iv = rsqrt_r(cabs2(a) + cabs2(bb));
        const cx<R> ah = cscale(iv, a), bh = cscale(iv, bb);
#pragma unroll
        for (int k = 0; k < M; k++) {
            if (k == j) {
                A[k][j] = csub(cmul(Ajj, bh), cmul(Bjj, ah));
            } else {
                const R sJ = s * J[k * NPHC_JSTRIDE + j];
                A[k][j] = cscale(sJ, cadd(cmul(y[k], bh), cmul(x[k], ah)));
            }
        }
#pragma unroll
        for (int r = 0; r < NR; r++) {
            const cx<R> q = cscale(iv, rg[r]);
            const cx<R> px = cmulc(ah, q), py = cmulc(bh, q);
#pragma unroll
            for (int k = 0; k < M; k++) {
                if (k == j) {
                    b[r][k] = csub(b[r][k], cadd(cmul(Ajj, px), cmul(Bjj, py)));
                } else {
                    const R sJ = s * J[k * NPHC_JSTRIDE + j];
                    b[r][k] = csub(b[r][k], cscale(sJ, csub(cmul(y[k], px), cmul(x[k], py))));
                }
            }
            b[r][j] = cadd(b[r][j], rf[r]);
        }
    }

    // ---- Householder QR: Q^H S = R (real diagonal), applied to the right-hand sides
    R dg[M];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < M; k++) {
        const cx<R> al = A[k][k];
        R xn2 = R(0);
#pragma unroll
        for (int i = k + 1; i < M; i++) xn2 += cabs2(A[i][k]);
        const R an = sqrt_r(cabs2(al) + xn2);
        ok = ok && (an > R(0));
        const R beta = al.re >= R(0) ? -an : an;
        const R ib = recip_r(beta);
        const cx<R> tauc = cx<R>{(beta - al.re) * ib, al.im * ib};   // conj(tau)
        const cx<R> sc = crecip(cx<R>{al.re - beta, al.im});
#pragma unroll
        for (int i = k + 1; i < M; i++) A[i][k] = cmul(A[i][k], sc);  // v_i (v_k = 1)
        dg[k] = beta;
#pragma unroll
        for (int c = k + 1; c < M; c++) {
            cx<R> wv = A[k][c];
#pragma unroll
            for (int i = k + 1; i < M; i++) wv = cadd(wv, cmulc(A[i][k], A[i][c]));
            wv = cmul(tauc, wv);
            A[k][c] = csub(A[k][c], wv);
#pragma unroll
            for (int i = k + 1; i < M; i++) A[i][c] = csub(A[i][c], cmul(A[i][k], wv));
        }
#pragma unroll
        for (int r = 0; r < NR; r++) {
            cx<R> wv = b[r][k];
#pragma unroll
            for (int i = k + 1; i < M; i++) wv = cadd(wv, cmulc(A[i][k], b[r][i]));
            wv = cmul(tauc, wv);
            b[r][k] = csub(b[r][k], wv);
#pragma unroll
            for (int i = k + 1; i < M; i++) b[r][i] = csub(b[r][i], cmul(A[i][k], wv));
        }
    }
    // back substitution R s = Q^H b (in place in b)
#pragma unroll
    for (int r = 0; r < NR; r++) {
#pragma unroll
        for (int k = M - 1; k >= 0; k--) {
            cx<R> acc = b[r][k];
#pragma unroll
            for (int c = k + 1; c < M; c++) acc = csub(acc, cmul(A[k][c], b[r][c]));
            b[r][k] = cscale(recip_r(dg[k]), acc);
        }
    }

    // ---- back to (dx, dy): reload the point rather than keep it live through the QR
    compiler_fence();
    R chk = R(0);
#pragma unroll
    for (int j = 0; j < M; j++) {
        const cx<R> xj = pt.get(j), yj = pt.get(M + j);
        const cx<R> a = cscale(R(2) * s, xj);
        const cx<R> bb = cscale(R(2), cmul(sg, yj));
        const R iv = rsqrt_r(cabs2(a) + cabs2(bb));
        const cx<R> ah = cscale(iv, a), bh = cscale(iv, bb);
        const cx<R> y2 = cmul(yj, yj), x2 = cmul(xj, xj);
        const cx<R> htg = csub(cmul(gam, cx<R>{y2.re - R(1), y2.im}),
                               cx<R>{x2.re + y2.re - R(1), x2.im + y2.im});
#pragma unroll
        for (int r = 0; r < NR; r++) {
            const cx<R> rg = (NR == 2 && r == 0) ? res.get(M + j) : htg;
            const cx<R> q = cscale(iv, rg);
            const cx<R> dx = cadd(cmulc(ah, q), cmul(bh, b[r][j]));
            const cx<R> dy = csub(cmulc(bh, q), cmul(ah, b[r][j]));
            chk += cabs2(dx) + cabs2(dy);
            if (wr) {
                const TVec<R, BLOCK> &o = (r == 0) ? out1 : out2;
                o.set(j, dx);
                o.set(M + j, dy);
            }
        }
    }
    return ok && finite_r(chk);
}

// -H(z, te) in the working precision R (no compensation), written to out when wr.
template <int M, class R, int BLOCK>
__device__ __forceinline__ void xy_residual_plain(const R *__restrict__ J, const TVec<R, BLOCK> &pt,
                                                  double te, cx<R> gam,
                                                  const TVec<R, BLOCK> &out, bool wr) {
    const R s = (R)te;
    const cx<R> gomt = cscale((R)(1.0 - te), gam);
    cx<R> x[M], y[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        x[k] = pt.get(k);
        y[k] = pt.get(M + k);
    }
#pragma unroll
    for (int k = 0; k < M; k++) {
        cx<R> u = cx<R>{J[k * NPHC_JSTRIDE + M], R(0)}, w = cx<R>{R(0), R(0)};
#pragma unroll
        for (int l = 0; l < M; l++) {
            if (l == k) continue;
            const R Jl = J[k * NPHC_JSTRIDE + l];
            u.re += Jl * x[l].re;
            u.im += Jl * x[l].im;
            w.re += Jl * y[l].re;
            w.im += Jl * y[l].im;
        }
        const cx<R> f = csub(cmul(y[k], u), cmul(x[k], w));
        const cx<R> x2 = cmul(x[k], x[k]), y2 = cmul(y[k], y[k]);
        const cx<R> hf = cadd(cmul(gomt, cx<R>{x2.re - R(1), x2.im}), cscale(s, f));
        const cx<R> hg = cadd(cmul(gomt, cx<R>{y2.re - R(1), y2.im}),
                              cscale(s, cx<R>{x2.re + y2.re - R(1), x2.im + y2.im}));
        if (wr) {
            out.set(k, cx<R>{-hf.re, -hf.im});
            out.set(M + k, cx<R>{-hg.re, -hg.im});
        }
    }
}

// -H(z, te) for an FP32 point, evaluated with compensated (float-float) sums and exact
// products, then rounded once: the error is ~2^-48 of the terms instead of 2^-24, so a
// Newton corrector driven by it converges to the FP32 rounding of the path point even
// when H_z is far from well conditioned (mixed-precision iterative refinement).  The
// coefficients J, gamma (1-t) and t enter as their FP32 values.
template <int M, int BLOCK>
__device__ __forceinline__ void xy_residual_ff(const float *__restrict__ J,
                                               const TVec<float, BLOCK> &pt, double te,
                                               cx<float> gam, const TVec<float, BLOCK> &out,
                                               bool wr) {
    const float s = (float)te;
    const float omt = (float)(1.0 - te);
    const cx<float> gomt = cx<float>{__fmul_rn(omt, gam.re), __fmul_rn(omt, gam.im)};
    cx<float> x[M], y[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        x[k] = pt.get(k);
        y[k] = pt.get(M + k);
    }
#pragma unroll
    for (int k = 0; k < M; k++) {
        ff ure = {J[k * NPHC_JSTRIDE + M], 0.f}, uim = {0.f, 0.f}, wre = {0.f, 0.f}, wim = {0.f, 0.f};
#pragma unroll
        for (int l = 0; l < M; l++) {
            if (l == k) continue;
            const float Jl = J[k * NPHC_JSTRIDE + l];
            ff_acc(ure, Jl, x[l].re);
            ff_acc(uim, Jl, x[l].im);
            ff_acc(wre, Jl, y[l].re);
            ff_acc(wim, Jl, y[l].im);
        }
        // f = y u - x w
        ff fre = {0.f, 0.f}, fim = {0.f, 0.f};
        ff_acc_ff(fre, y[k].re, ure);
        ff_acc_ff(fre, -y[k].im, uim);
        ff_acc_ff(fre, -x[k].re, wre);
        ff_acc_ff(fre, x[k].im, wim);
        ff_acc_ff(fim, y[k].re, uim);
        ff_acc_ff(fim, y[k].im, ure);
        ff_acc_ff(fim, -x[k].re, wim);
        ff_acc_ff(fim, -x[k].im, wre);
        // x^2 - 1, y^2 - 1 and c^2 + s^2 - 1, exactly as float-float
        ff qxr = {-1.f, 0.f}, qxi = {0.f, 0.f}, qyr = {-1.f, 0.f}, qyi = {0.f, 0.f};
        ff_acc(qxr, x[k].re, x[k].re);
        ff_acc(qxr, -x[k].im, x[k].im);
        ff_acc(qxi, 2.f * x[k].re, x[k].im);
        ff_acc(qyr, y[k].re, y[k].re);
        ff_acc(qyr, -y[k].im, y[k].im);
        ff_acc(qyi, 2.f * y[k].re, y[k].im);
        // H_f = gomt (x^2 - 1) + s f ;  H_g = gomt (y^2 - 1) + s (x^2 + y^2 - 1)
        ff hfr = {0.f, 0.f}, hfi = {0.f, 0.f}, hgr = {0.f, 0.f}, hgi = {0.f, 0.f};
        ff_acc_ff(hfr, gomt.re, qxr);
        ff_acc_ff(hfr, -gomt.im, qxi);
        ff_acc_ff(hfr, s, fre);
        ff_acc_ff(hfi, gomt.re, qxi);
        ff_acc_ff(hfi, gomt.im, qxr);
        ff_acc_ff(hfi, s, fim);
        ff_acc_ff(hgr, gomt.re, qyr);
        ff_acc_ff(hgr, -gomt.im, qyi);
        ff_acc_ff(hgr, s, qxr);
        ff_acc_ff(hgr, s, qyr);
        ff_acc(hgr, s, 1.f);       // x^2 + y^2 - 1 = (x^2 - 1) + (y^2 - 1) + 1
        ff_acc_ff(hgi, gomt.re, qyi);
        ff_acc_ff(hgi, gomt.im, qyr);
        ff_acc_ff(hgi, s, qxi);
        ff_acc_ff(hgi, s, qyi);
        if (wr) {
            out.set(k, cx<float>{-ff_val(hfr), -ff_val(hfi)});
            out.set(M + k, cx<float>{-ff_val(hgr), -ff_val(hgi)});
        }
    }
}
