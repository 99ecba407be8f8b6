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
// where A = d(f rows)/dx and B = d(f rows)/dy of H.  S is solved by Householder QR:
// unitary (no pivot search, no growth) and data-independent in its control flow.
// Cost ~ (8/3) M^3 + O(M^2 + M N) real flops instead of (8/3) (2M)^3 for the full system.
//
// Memory layout (one path per thread): the augmented M x (M + 2) matrix [S | b0 | b1]
// of each thread lives in shared memory, column-major, each complex entry interleaved
// across the threads of the block (entry (i, c) of thread t at [(c M + i) BLOCK + t]:
// conflict-free 64-bit accesses).  The Householder step k is a runtime loop: its
// reflector sits in registers, and the remaining columns, right-hand sides included,
// stream through registers one at a time in a loop of fixed length M that leaves early
// (k is the same for every thread of a warp, so the exit is uniform).  The QR, the back
// substitution and the recovery thus each exist once in the code: unrolled over k they
// outgrow the instruction cache from M ~ 8 on, and the kernel stalls on instruction
// fetch.
#pragma once

#include "nphc_internal.cuh"

// One thread's vector of 2M complex unknowns in shared memory, interleaved across the
// threads of the block (element i of thread t at [i * BLOCK + t]).
template <class R, int BLOCK>
struct SVec {
    cx<R> *p;
    __device__ __forceinline__ cx<R> get(int i) const { return p[i * BLOCK]; }
    __device__ __forceinline__ void set(int i, cx<R> v) const { p[i * BLOCK] = v; }
};

// One thread's vector in global scratch (element i at [i * stride]); stride = threads in
// the grid, so a warp's accesses are coalesced.
template <class R>
struct GVec {
    cx<R> *p;
    int64_t stride;
    __device__ __forceinline__ cx<R> get(int i) const { return p[i * stride]; }
    __device__ __forceinline__ void set(int i, cx<R> v) const { p[i * stride] = v; }
};

// One thread's M x M complex matrix in shared memory, column-major.
template <int M, class R, int BLOCK>
struct SMat {
    cx<R> *p;
    __device__ __forceinline__ cx<R> get(int i, int c) const { return p[(c * M + i) * BLOCK]; }
    __device__ __forceinline__ void set(int i, int c, cx<R> v) const { p[(c * M + i) * BLOCK] = v; }
};

// Shared memory per thread: the augmented matrix plus the evaluation point.  The solve's
// output / residual vector (2M entries) shares the matrix's two right-hand-side columns
// (also 2M entries, column-major and contiguous): the solve consumes a residual there
// while it builds S, before it writes the right-hand sides, and it reads each solution
// entry before it writes the output entry in the same place.  Seven 32-thread blocks
// per SM fit at M = 9 instead of six.
template <int M, class R>
constexpr size_t xy_smem_per_thread() { return sizeof(cx<R>) * (size_t)(M * (M + 2) + 2 * M); }

__device__ __forceinline__ void compiler_fence() { asm volatile("" ::: "memory"); }

// -H_t rows of site k (H_t = P - gamma Q) at the point (xk, yk) with u_k, w_k given.
template <class R>
__device__ __forceinline__ void minus_ht_rows(cx<R> xk, cx<R> yk, cx<R> u, cx<R> w, cx<R> gam,
                                              cx<R> &rf, cx<R> &rg) {
    const cx<R> f = csub(cmul(yk, u), cmul(xk, w));
    const cx<R> x2 = cmul(xk, xk), y2 = cmul(yk, yk);
    rf = csub(cmul(gam, cx<R>{x2.re - R(1), x2.im}), f);
    rg = csub(cmul(gam, cx<R>{y2.re - R(1), y2.im}), cx<R>{x2.re + y2.re - R(1), x2.im + y2.im});
}

// -H_t constraint row only (needs no couplings).
template <class R>
__device__ __forceinline__ cx<R> minus_ht_g(cx<R> xk, cx<R> yk, cx<R> gam) {
    const cx<R> x2 = cmul(xk, xk), y2 = cmul(yk, yk);
    return csub(cmul(gam, cx<R>{y2.re - R(1), y2.im}), cx<R>{x2.re + y2.re - R(1), x2.im + y2.im});
}

// u_k = J_{k,N} + sum_l J_kl x_l and w_k = sum_l J_kl y_l (J_kk = 0, so the sum may run over
// every l).  k may be a runtime index (the row of J is then read with a uniform offset).
template <int M, class R>
__device__ __forceinline__ void xy_uw(const R *__restrict__ J, const cx<R> (&x)[M],
                                      const cx<R> (&y)[M], int k, cx<R> &u, cx<R> &w) {
    const R *Jk = J + k * NPHC_JSTRIDE;
    u = cx<R>{Jk[M], R(0)};
    w = cx<R>{R(0), R(0)};
#pragma unroll
    for (int l = 0; l < M; l++) {
        const R Jl = Jk[l];
        u.re += Jl * x[l].re;
        u.im += Jl * x[l].im;
        w.re += Jl * y[l].re;
        w.im += Jl * y[l].im;
    }
}

// Frame of constraint row j: (a^, b^) and 1 / |(a_j, b_j)|.
template <class R>
__device__ __forceinline__ void g_frame(cx<R> xj, cx<R> yj, R s, cx<R> sg, cx<R> &ah, cx<R> &bh,
                                        R &iv) {
    const cx<R> a = cscale(R(2) * s, xj);
    const cx<R> bb = cscale(R(2), cmul(sg, yj));
    iv = rsqrt_r(cabs2(a) + cabs2(bb));
    ah = cscale(iv, a);
    bh = cscale(iv, bb);
}

// Solve S x = b for the M x M matrix S of an augmented per-thread matrix
// [S | b0 | b1] (b1 only when two_rhs) by Householder QR: Q^H [S | b] = [R | Q^H b] with a
// real diagonal (stored as (beta, 0) on the diagonal of S), then back substitution in
// place: the solutions end in columns M and M + 1.  Returns false when S is singular.
template <int M, class R, int BLOCK>
__device__ __forceinline__ bool aug_qr_solve(const SMat<M, R, BLOCK> &A, bool two_rhs) {
    const int ncol = two_rhs ? M + 2 : M + 1;
    bool ok = true;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const int n = M - k;   // active rows k .. M-1, relative index i = 0 .. n-1
        const SMat<M, R, BLOCK> Ak{A.p + k * BLOCK};   // Ak.get(i, c) = S(k + i, c)
        // loads first, then arithmetic (all shared loads of a column in flight at once),
        // sums split in two chains
        cx<R> v[M];
        const cx<R> al = Ak.get(0, k);
#pragma unroll
        for (int i = 1; i < M; i++) {
            if (i >= n) break;
            v[i] = Ak.get(i, k);
        }
        R xa = R(0), xb = R(0);
#pragma unroll
        for (int i = 1; i < M; i++) {
            if (i >= n) break;
            if (i & 1) xa += cabs2(v[i]);
            else xb += cabs2(v[i]);
        }
        const R an = sqrt_r(cabs2(al) + (xa + xb));
        ok = ok && (an > R(0));
        const R beta = al.re >= R(0) ? -an : an;
        const R ib = recip_r(beta);
        const cx<R> tauc = cx<R>{(beta - al.re) * ib, al.im * ib};   // conj(tau)
        const cx<R> sc = crecip(cx<R>{al.re - beta, al.im});
#pragma unroll
        for (int i = 1; i < M; i++) {
            if (i >= n) break;
            v[i] = cmul(v[i], sc);   // reflector (1, v_1, .., v_{n-1})
        }
        Ak.set(0, k, cx<R>{beta, R(0)});
#pragma unroll 1
        for (int c = k + 1; c < ncol; c++) {
            cx<R> col[M];
#pragma unroll
            for (int i = 0; i < M; i++) {
                if (i >= n) break;
                col[i] = Ak.get(i, c);
            }
            cx<R> wa = col[0], wb = cx<R>{R(0), R(0)};
#pragma unroll
            for (int i = 1; i < M; i++) {
                if (i >= n) break;
                if (i & 1) wb = cadd(wb, cmulc(v[i], col[i]));
                else wa = cadd(wa, cmulc(v[i], col[i]));
            }
            const cx<R> wv = cmul(tauc, cadd(wa, wb));
            Ak.set(0, c, csub(col[0], wv));
#pragma unroll
            for (int i = 1; i < M; i++) {
                if (i >= n) break;
                Ak.set(i, c, csub(col[i], cmul(v[i], wv)));
            }
        }
    }

    // ---- back substitution R s = Q^H b, column by column, in place in columns M, M + 1
#pragma unroll 1
    for (int k = M - 1; k >= 0; k--) {
        const R ir = recip_r(A.get(k, k).re);
        const cx<R> s0 = cscale(ir, A.get(k, M));
        A.set(k, M, s0);
        cx<R> s1 = cx<R>{R(0), R(0)};
        if (two_rhs) {
            s1 = cscale(ir, A.get(k, M + 1));
            A.set(k, M + 1, s1);
        }
        constexpr int MA = M > 1 ? M - 1 : 1;
        cx<R> Rc[MA], c0[MA], c1[MA];
#pragma unroll
        for (int i = 0; i < M - 1; i++) {
            if (i >= k) break;
            Rc[i] = A.get(i, k);
            c0[i] = A.get(i, M);
            if (two_rhs) c1[i] = A.get(i, M + 1);
        }
#pragma unroll
        for (int i = 0; i < M - 1; i++) {
            if (i >= k) break;
            A.set(i, M, csub(c0[i], cmul(Rc[i], s0)));
            if (two_rhs) A.set(i, M + 1, csub(c1[i], cmul(Rc[i], s1)));
        }
    }

    return ok;
}

// Solve H_z(z, t) d = r at the point in `pt`, with t given as (s, omt) = (t, 1 - t).
//   two_rhs == false: r = -H_t (predictor: d = dz/dt), written to out1.
//   two_rhs == true:  r1 = the residual vector in `res` (corrector: -H), written to out1;
//                     r2 = -H_t, written to out2.
// res and out1 may be the matrix's right-hand-side columns (see xy_smem_per_thread); the
// residual's g rows, needed again after the factorisation, wait in out2 meanwhile.
// two_rhs must be uniform across the warp.  Outputs are written only when wr.  Returns
// false when the system is singular or the result is not finite.
template <int M, class R, int BLOCK, class Out2>
__device__ __forceinline__ bool xy_solve(const R *__restrict__ J, const SMat<M, R, BLOCK> &A,
                                         const SVec<R, BLOCK> &pt, R s, R omt, cx<R> gam,
                                         bool two_rhs, const SVec<R, BLOCK> &res,
                                         const SVec<R, BLOCK> &out1, const Out2 &out2, bool wr) {
    const cx<R> gomt = cscale(omt, gam);
    const cx<R> sg = cx<R>{s + gomt.re, gomt.im};   // t + gamma (1 - t)

    cx<R> x[M], y[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        x[k] = pt.get(k);
        y[k] = pt.get(M + k);
    }
    cx<R> b0[M], b1[M];
#pragma unroll
    for (int k = 0; k < M; k++) b0[k] = b1[k] = cx<R>{R(0), R(0)};

    // ---- build S column by column (columns j in a loop; rows unrolled)
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        const cx<R> xj = pt.get(j), yj = pt.get(M + j);
        cx<R> u, w, htf, htg;
        xy_uw<M, R>(J, x, y, j, u, w);
        minus_ht_rows<R>(xj, yj, u, w, gam, htf, htg);
        const cx<R> rf0 = two_rhs ? res.get(j) : htf;
        const cx<R> rg0 = two_rhs ? res.get(M + j) : htg;
        // diagonal Jacobian entries of gradient row j
        const cx<R> Ajj = cx<R>{-s * w.re + R(2) * (gomt.re * xj.re - gomt.im * xj.im),
                                -s * w.im + R(2) * (gomt.re * xj.im + gomt.im * xj.re)};
        const cx<R> Bjj = cscale(s, u);
        cx<R> ah, bh;
        R iv;
        g_frame<R>(xj, yj, s, sg, ah, bh, iv);
        const cx<R> q0 = cscale(iv, rg0), q1 = cscale(iv, htg);
        const cx<R> px0 = cmulc(ah, q0), py0 = cmulc(bh, q0);
        const cx<R> px1 = cmulc(ah, q1), py1 = cmulc(bh, q1);
        // the diagonal's own contributions, added to row j below
        const cx<R> d0 = csub(rf0, cadd(cmul(Ajj, px0), cmul(Bjj, py0)));
        const cx<R> d1 = csub(htf, cadd(cmul(Ajj, px1), cmul(Bjj, py1)));
        if (two_rhs && wr) out2.set(M + j, rg0);   // the residual's g row, for the recovery
#pragma unroll
        for (int k = 0; k < M; k++) {
            // off-diagonal entries; J_jj = 0 makes the k == j term vanish
            const R sJ = s * J[k * NPHC_JSTRIDE + j];
            A.set(k, j, cscale(sJ, cadd(cmul(y[k], bh), cmul(x[k], ah))));
            b0[k] = csub(b0[k], cscale(sJ, csub(cmul(y[k], px0), cmul(x[k], py0))));
            if (two_rhs) b1[k] = csub(b1[k], cscale(sJ, csub(cmul(y[k], px1), cmul(x[k], py1))));
            if (k == j) {
                b0[k] = cadd(b0[k], d0);
                b1[k] = cadd(b1[k], d1);
            }
        }
        A.set(j, j, csub(cmul(Ajj, bh), cmul(Bjj, ah)));
    }

    // right-hand sides into columns M and M + 1
#pragma unroll
    for (int k = 0; k < M; k++) {
        A.set(k, M, b0[k]);
        if (two_rhs) A.set(k, M + 1, b1[k]);
    }

    bool ok = aug_qr_solve<M, R, BLOCK>(A, two_rhs);

    // ---- back to (dx, dy)
    R chk = R(0);
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        const cx<R> xj = pt.get(j), yj = pt.get(M + j);
        cx<R> ah, bh;
        R iv;
        g_frame<R>(xj, yj, s, sg, ah, bh, iv);
        const cx<R> htg = minus_ht_g<R>(xj, yj, gam);
        const cx<R> q0 = cscale(iv, two_rhs ? out2.get(M + j) : htg);
        const cx<R> s0 = A.get(j, M);
        const cx<R> dx0 = cadd(cmulc(ah, q0), cmul(bh, s0));
        const cx<R> dy0 = csub(cmulc(bh, q0), cmul(ah, s0));
        chk += cabs2(dx0) + cabs2(dy0);
        if (two_rhs) {
            const cx<R> q1 = cscale(iv, htg);
            const cx<R> s1 = A.get(j, M + 1);
            const cx<R> dx1 = cadd(cmulc(ah, q1), cmul(bh, s1));
            const cx<R> dy1 = csub(cmulc(bh, q1), cmul(ah, s1));
            chk += cabs2(dx1) + cabs2(dy1);
            if (wr) {
                out2.set(j, dx1);
                out2.set(M + j, dy1);
            }
        }
        if (wr) {
            out1.set(j, dx0);
            out1.set(M + j, dy0);
        }
    }
    return ok && finite_r(chk);
}

// -H(z, t) in the working precision R (no compensation), written to out when wr.
template <int M, class R, int BLOCK>
__device__ __forceinline__ void xy_residual_plain(const R *__restrict__ J, const SVec<R, BLOCK> &pt,
                                                  R s, R omt, cx<R> gam,
                                                  const SVec<R, BLOCK> &out, bool wr) {
    const cx<R> gomt = cscale(omt, gam);
    cx<R> x[M], y[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        x[k] = pt.get(k);
        y[k] = pt.get(M + k);
    }
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const cx<R> xk = pt.get(k), yk = pt.get(M + k);
        cx<R> u, w;
        xy_uw<M, R>(J, x, y, k, u, w);
        const cx<R> f = csub(cmul(yk, u), cmul(xk, w));
        const cx<R> x2 = cmul(xk, xk), y2 = cmul(yk, yk);
        const cx<R> hf = cadd(cmul(gomt, cx<R>{x2.re - R(1), x2.im}), cscale(s, f));
        const cx<R> hg = cadd(cmul(gomt, cx<R>{y2.re - R(1), y2.im}),
                              cscale(s, cx<R>{x2.re + y2.re - R(1), x2.im + y2.im}));
        if (wr) {
            out.set(k, cx<R>{-hf.re, -hf.im});
            out.set(M + k, cx<R>{-hg.re, -hg.im});
        }
    }
}

// -H(z, t) evaluated with compensated sums (float-float for FP32, double-double for
// FP64) and exact products, then rounded once: the error is ~u^2 of the terms instead of
// u, so a Newton corrector driven by it converges to the rounding of the path point
// even when H_z is far from well conditioned (mixed-precision iterative refinement; at
// large ||z|| the terms of H are ~||z||^2 while H itself is near zero).  The coefficients
// J, gamma (1-t) and t enter as their values in R.
template <int M, class R, int BLOCK>
__device__ __forceinline__ void xy_residual_comp(const R *__restrict__ J,
                                                 const SVec<R, BLOCK> &pt, R s, R omt,
                                                 cx<R> gam, const SVec<R, BLOCK> &out, bool wr) {
    using E = EFT<R>;
    const cx<R> gomt = cx<R>{E::mul(omt, gam.re), E::mul(omt, gam.im)};
    cx<R> x[M], y[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        x[k] = pt.get(k);
        y[k] = pt.get(M + k);
    }
    const ext<R> zero = {R(0), R(0)};
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const cx<R> xk = pt.get(k), yk = pt.get(M + k);
        const R *Jk = J + k * NPHC_JSTRIDE;
        ext<R> ure = {Jk[M], R(0)}, uim = zero, wre = zero, wim = zero;
#pragma unroll
        for (int l = 0; l < M; l++) {   // J_kk = 0 adds exact zeros
            const R Jl = Jk[l];
            ext_acc(ure, Jl, x[l].re);
            ext_acc(uim, Jl, x[l].im);
            ext_acc(wre, Jl, y[l].re);
            ext_acc(wim, Jl, y[l].im);
        }
        // f = y u - x w
        ext<R> fre = zero, fim = zero;
        ext_acc_ext(fre, yk.re, ure);
        ext_acc_ext(fre, -yk.im, uim);
        ext_acc_ext(fre, -xk.re, wre);
        ext_acc_ext(fre, xk.im, wim);
        ext_acc_ext(fim, yk.re, uim);
        ext_acc_ext(fim, yk.im, ure);
        ext_acc_ext(fim, -xk.re, wim);
        ext_acc_ext(fim, -xk.im, wre);
        // x^2 - 1 and y^2 - 1 exactly as two-word numbers
        ext<R> qxr = {R(-1), R(0)}, qxi = zero, qyr = {R(-1), R(0)}, qyi = zero;
        ext_acc(qxr, xk.re, xk.re);
        ext_acc(qxr, -xk.im, xk.im);
        ext_acc(qxi, R(2) * xk.re, xk.im);
        ext_acc(qyr, yk.re, yk.re);
        ext_acc(qyr, -yk.im, yk.im);
        ext_acc(qyi, R(2) * yk.re, yk.im);
        // H_f = gomt (x^2 - 1) + s f ;  H_g = gomt (y^2 - 1) + s (x^2 + y^2 - 1)
        ext<R> hfr = zero, hfi = zero, hgr = zero, hgi = zero;
        ext_acc_ext(hfr, gomt.re, qxr);
        ext_acc_ext(hfr, -gomt.im, qxi);
        ext_acc_ext(hfr, s, fre);
        ext_acc_ext(hfi, gomt.re, qxi);
        ext_acc_ext(hfi, gomt.im, qxr);
        ext_acc_ext(hfi, s, fim);
        ext_acc_ext(hgr, gomt.re, qyr);
        ext_acc_ext(hgr, -gomt.im, qyi);
        ext_acc_ext(hgr, s, qxr);
        ext_acc_ext(hgr, s, qyr);
        ext_acc(hgr, s, R(1));       // x^2 + y^2 - 1 = (x^2 - 1) + (y^2 - 1) + 1
        ext_acc_ext(hgi, gomt.re, qyi);
        ext_acc_ext(hgi, gomt.im, qyr);
        ext_acc_ext(hgi, s, qxi);
        ext_acc_ext(hgi, s, qyi);
        if (wr) {
            out.set(k, cx<R>{-ext_val(hfr), -ext_val(hfi)});
            out.set(M + k, cx<R>{-ext_val(hgr), -ext_val(hgi)});
        }
    }
}
