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
// Each site's step is written in scaled light-cone coordinates: with p_k = x_k + i y_k,
// q_k = x_k - i y_k (e^(+-i theta_k) on the real circle), sp = max(1, |p_k|),
// sq = max(1, |q_k|),
//   dx_k = (sp dwp_k + sq dwq_k) / 2,   dy_k = -i (sp dwp_k - sq dwq_k) / 2,
// so a row's coefficients (al, be) on (dx_k, dy_k) become (sp (al - i be) / 2,
// sq (al + i be) / 2) on (dwp_k, dwq_k).  On a path to infinity one of p_k, q_k grows
// like ||z|| while the other shrinks, and in (x, y) the Jacobian's condition number grows
// like ||z||^2; in the scaled coordinates it stays moderate (measured on the N = 10 ring
// at ||z|| = 1e8: a median of 1e4.5 against 1e13), so FP32 can follow a path to a finite
// solution of large norm, or to the divergence radius.  At ||z|| <= 1 the scales are 1 and
// the change is sqrt(1/2) times a unitary one.
// A unitary change of variables per site, (dwp_k, dwq_k) = conj(a^, b^) q_k + (b^, -a^) s_k
// with (a^, b^) the constraint row's coefficients (a'_k, b'_k) on (dwp_k, dwq_k) over their
// norm, turns that row into q_k = r_gk / |(a'_k, b'_k)| and leaves an M x M complex system
// for s in the gradient rows:
//   S_kj = A'_kj b^_j - B'_kj a^_j,   rhs_k = r_fk - sum_j (A'_kj conj(a^_j) + B'_kj conj(b^_j)) q_j,
// where A', B' are the gradient rows' coefficients on dwp_j, dwq_j.  For k != j
// (A_kj, B_kj) = t J_kj (y_k, -x_k), which become (i t J_kj / 2) (sp_j q_k, -sq_j p_k).  S is
// solved by LU with partial pivoting (aug_lu_solve; the generic quadratic systems use the
// Householder QR, aug_qr_solve): its control flow is data-independent too (the pivot is
// a per-thread row index, the loops run the same for every thread), and its column sweep
// costs about 6 instructions per complex entry against Householder's 10 (measured on the
// N = 10 ring: the FP32 pass 134 -> 117 ms with the same solve count).  Cost ~ (8/3) M^3
// + O(M^2 + M N) real flops instead of (8/3) (2M)^3 for the full system.
//
// Memory layout (one path per thread): the augmented M x (M + 2) matrix [S | b0 | b1]
// of each thread lives in shared memory, column-major, each complex entry interleaved
// across the threads of the block (entry (i, c) of thread t at [(c M + i) BLOCK + t]:
// conflict-free 64-bit accesses).  The elimination step k is a runtime loop: its
// reflector or multipliers sit in registers, and the remaining columns, right-hand sides
// included, stream through registers one at a time in a loop of fixed length M that leaves
// early (k is the same for every thread of a warp, so the exit is uniform).  The
// factorisation, the back substitution and the recovery thus each exist once in the code:
// unrolled over k they
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

// Coefficients (al, be) of a row on (dx_j, dy_j) as coefficients on the scaled light-cone
// step (dwp_j, dwq_j): (sp (al - i be) / 2, sq (al + i be) / 2).
template <class R>
__device__ __forceinline__ void lc_coef(cx<R> al, cx<R> be, R sp, R sq, cx<R> &alp, cx<R> &bep) {
    alp = cscale(R(0.5) * sp, cx<R>{al.re + be.im, al.im - be.re});
    bep = cscale(R(0.5) * sq, cx<R>{al.re - be.im, al.im + be.re});
}

// Scales of site j's light-cone coordinates: max(1, |x + i y|) and max(1, |x - i y|).
template <class R>
__device__ __forceinline__ void lc_scales(cx<R> xj, cx<R> yj, R &sp, R &sq) {
    const cx<R> p = cx<R>{xj.re - yj.im, xj.im + yj.re}, q = cx<R>{xj.re + yj.im, xj.im - yj.re};
    sp = fmax(R(1), sqrt_r(cabs2(p)));
    sq = fmax(R(1), sqrt_r(cabs2(q)));
}

// Frame of constraint row j in site j's scaled light-cone coordinates: (a^, b^), the
// inverse of the row's norm |(a'_j, b'_j)| and the scales sp, sq.
template <class R>
__device__ __forceinline__ void g_frame(cx<R> xj, cx<R> yj, R s, cx<R> sg, cx<R> &ah, cx<R> &bh,
                                        R &iv, R &sp, R &sq) {
    lc_scales<R>(xj, yj, sp, sq);
    cx<R> a, bb;
    lc_coef<R>(cscale(R(2) * s, xj), cscale(R(2), cmul(sg, yj)), sp, sq, a, bb);
    iv = rsqrt_r(cabs2(a) + cabs2(bb));
    ah = cscale(iv, a);
    bh = cscale(iv, bb);
}

// (dx_j, dy_j) from the light-cone step (dwp, dwq) = conj(a^, b^) q + (b^, -a^) s.
template <class R>
__device__ __forceinline__ void lc_step(cx<R> ah, cx<R> bh, R sp, R sq, cx<R> q, cx<R> s,
                                        cx<R> &dx, cx<R> &dy) {
    const cx<R> wp = cscale(sp, cadd(cmulc(ah, q), cmul(bh, s)));
    const cx<R> wq = cscale(sq, csub(cmulc(bh, q), cmul(ah, s)));
    dx = cscale(R(0.5), cadd(wp, wq));
    const cx<R> d = csub(wp, wq);
    dy = cx<R>{R(0.5) * d.im, R(-0.5) * d.re};   // -i (wp - wq) / 2
}

// i c
template <class R>
__device__ __forceinline__ cx<R> cmul_i(cx<R> c) { return cx<R>{-c.im, c.re}; }

// Solve S x = b for the M x M matrix S of an augmented per-thread matrix
// [S | b0 | b1] (b1 only when two_rhs) by Householder QR: Q^H [S | b] = [R | Q^H b] with a
// real diagonal (stored as (beta, 0) on the diagonal of S), then back substitution in
// place: the solutions end in columns M and M + 1.  Returns false when S is singular.
// kest (may be NULL) receives max_k |R_kk| / min_k |R_kk|, a lower bound on the condition
// number of S that costs two comparisons per column.
template <int M, class R, int BLOCK>
__device__ __forceinline__ bool aug_qr_solve(const SMat<M, R, BLOCK> &A, bool two_rhs,
                                             R *kest = nullptr) {
    const int ncol = two_rhs ? M + 2 : M + 1;
    bool ok = true;
    R rmax = R(0), rmin = R(0);
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
        rmax = fmax(rmax, an);
        rmin = k == 0 ? an : fmin(rmin, an);
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

    if (kest) *kest = rmin > R(0) ? rmax / rmin : R(INFINITY);
    return ok;
}

// The same solve by LU with partial pivoting: per column one pivot search (the largest
// |a|^2 at or below the diagonal), one complex reciprocal, the multipliers in registers;
// then each trailing column (right-hand sides included) streams through once: rows k and
// p are swapped in shared memory (two loads, two stores at a per-thread index, still
// conflict-free in the interleaved layout) and the rows below take a rank-one update,
// a load, four FMAs and a store per complex entry, against Householder's extra dot
// product per entry.  The pivot's reciprocal replaces U_kk for the back substitution.
// kest (may be NULL) receives max_k |U_kk| / min_k |U_kk|, the usual cheap estimate of the
// condition number from a pivoted factorisation.
template <int M, class R, int BLOCK>
__device__ __forceinline__ bool aug_lu_solve(const SMat<M, R, BLOCK> &A, bool two_rhs,
                                             R *kest = nullptr) {
    const int ncol = two_rhs ? M + 2 : M + 1;
    bool ok = true;
    R umax = R(0), umin = R(0);
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const int n = M - k;   // active rows k .. M-1, relative index i = 0 .. n-1
        const SMat<M, R, BLOCK> Ak{A.p + k * BLOCK};   // Ak.get(i, c) = S(k + i, c)
        cx<R> v[M];
        cx<R> piv = Ak.get(0, k);
        R best = cabs2(piv);
        int p = 0;
        v[0] = piv;
#pragma unroll
        for (int i = 1; i < M; i++) {
            if (i >= n) break;
            v[i] = Ak.get(i, k);
            const R m = cabs2(v[i]);
            if (m > best) {
                best = m;
                p = i;
                piv = v[i];
            }
        }
        ok = ok && (best > R(0));
        const R um = sqrt_r(best);
        umax = fmax(umax, um);
        umin = k == 0 ? um : fmin(umin, um);
        const cx<R> ip = crecip(piv);
        // multipliers of rows 1 .. n-1 after the swap (row p holds the old row k)
#pragma unroll
        for (int i = 1; i < M; i++) {
            if (i >= n) break;
            v[i] = cmul(i == p ? v[0] : v[i], ip);
        }
        Ak.set(0, k, ip);
#pragma unroll 1
        for (int c = k + 1; c < ncol; c++) {
            const cx<R> a0 = Ak.get(0, c), ap = Ak.get(p, c);
            Ak.set(p, c, a0);
            Ak.set(0, c, ap);
#pragma unroll
            for (int i = 1; i < M; i++) {
                if (i >= n) break;
                const cx<R> x = Ak.get(i, c), l = v[i];
                Ak.set(i, c, cx<R>{fma(l.im, ap.im, fma(-l.re, ap.re, x.re)),
                                   fma(-l.im, ap.re, fma(-l.re, ap.im, x.im))});
            }
        }
    }

    // ---- back substitution U s = b, column by column, in place in columns M, M + 1
#pragma unroll 1
    for (int k = M - 1; k >= 0; k--) {
        const cx<R> ir = A.get(k, k);   // 1 / U_kk
        const cx<R> s0 = cmul(A.get(k, M), ir);
        A.set(k, M, s0);
        cx<R> s1 = cx<R>{R(0), R(0)};
        if (two_rhs) {
            s1 = cmul(A.get(k, M + 1), ir);
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

    if (kest) *kest = umin > R(0) ? umax / umin : R(INFINITY);
    return ok;
}

// ------------------------------------------------------------------------------------
// The per-thread trackers keep each site's unknowns in light-cone coordinates,
// p_k = x_k + i y_k and q_k = x_k - i y_k (the pinned site has p_N = q_N = 1).  Near infinity
// one of them is tiny next to x_k and y_k, so (x, y) in FP32 would lose it to cancellation
// once 1 - t < ~1e-6; in (p, q) the equations keep it exactly:
//   f_k = -i (p_k U_q,k - q_k U_p,k) / 2,  U_p,k = sum_j J_kj p_j,  U_q,k = sum_j J_kj q_j,
//   g_k = p_k q_k - 1,  x_k^2 - 1 = (p_k + q_k)^2 / 4 - 1,  y_k^2 - 1 = -(p_k - q_k)^2 / 4 - 1
// (sums over every other site, the pinned one included).  The step is (dp, dq) =
// (sp dwp, sq dwq), the scaled light-cone step of the solve above.

// U_p,k and U_q,k (J_kk = 0, so the sums may run over every l); k may be a runtime index.
template <int M, class R>
__device__ __forceinline__ void lc_U(const R *__restrict__ J, const cx<R> (&p)[M],
                                     const cx<R> (&q)[M], int k, cx<R> &Up, cx<R> &Uq) {
    const R *Jk = J + k * NPHC_JSTRIDE;
    Up = cx<R>{Jk[M], R(0)};
    Uq = Up;
#pragma unroll
    for (int l = 0; l < M; l++) {
        const R Jl = Jk[l];
        Up.re += Jl * p[l].re;
        Up.im += Jl * p[l].im;
        Uq.re += Jl * q[l].re;
        Uq.im += Jl * q[l].im;
    }
}

// -H_t rows of site k (H_t = P - gamma Q) in light-cone coordinates.
template <class R>
__device__ __forceinline__ void lc_minus_ht_rows(cx<R> pk, cx<R> qk, cx<R> Up, cx<R> Uq,
                                                 cx<R> gam, cx<R> &rf, cx<R> &rg) {
    const cx<R> f = cscale(R(0.5), cmul_i(csub(cmul(qk, Up), cmul(pk, Uq))));
    const cx<R> a = cadd(pk, qk), d = csub(pk, qk);
    const cx<R> a2 = cmul(a, a), d2 = cmul(d, d), g = cmul(pk, qk);
    rf = csub(cmul(gam, cx<R>{R(0.25) * a2.re - R(1), R(0.25) * a2.im}), f);
    rg = csub(cmul(gam, cx<R>{R(-0.25) * d2.re - R(1), R(-0.25) * d2.im}), cx<R>{g.re - R(1), g.im});
}

// -H_t constraint row only (needs no couplings).
template <class R>
__device__ __forceinline__ cx<R> lc_minus_ht_g(cx<R> pk, cx<R> qk, cx<R> gam) {
    const cx<R> d = csub(pk, qk);
    const cx<R> d2 = cmul(d, d), g = cmul(pk, qk);
    return csub(cmul(gam, cx<R>{R(-0.25) * d2.re - R(1), R(-0.25) * d2.im}), cx<R>{g.re - R(1), g.im});
}

// Frame of constraint row j at the light-cone point (p, q): the row's coefficients on
// (dwp, dwq) are (sp (t q - gamma (1-t) (p - q) / 2), sq (t p + gamma (1-t) (p - q) / 2)).
template <class R>
__device__ __forceinline__ void g_frame_lc(cx<R> pj, cx<R> qj, R s, cx<R> gomt, cx<R> &ah,
                                           cx<R> &bh, R &iv, R &sp, R &sq) {
    sp = fmax(R(1), sqrt_r(cabs2(pj)));
    sq = fmax(R(1), sqrt_r(cabs2(qj)));
    const cx<R> hd = cscale(R(0.5), cmul(gomt, csub(pj, qj)));
    const cx<R> a = cscale(sp, csub(cscale(s, qj), hd));
    const cx<R> b = cscale(sq, cadd(cscale(s, pj), hd));
    iv = rsqrt_r(cabs2(a) + cabs2(b));
    ah = cscale(iv, a);
    bh = cscale(iv, b);
}

// Solve H_z(z, t) d = r at the light-cone point in `pt` (p_1..p_M, q_1..q_M), t given as
// (s, omt) = (t, 1 - t); d is the light-cone step (dp, dq).
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
                                         const SVec<R, BLOCK> &out1, const Out2 &out2, bool wr,
                                         R *kest = nullptr) {
    const cx<R> gomt = cscale(omt, gam);

    cx<R> p[M], q[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        p[k] = pt.get(k);
        q[k] = pt.get(M + k);
    }
    // right-hand sides as sums over the columns: b_k = d_k - (i t / 2) (q_k sum_j J_kj X_j -
    // p_k sum_j J_kj Y_j), X_j = sp_j conj(a^_j) q_j, Y_j = sq_j conj(b^_j) q_j, d_k the
    // diagonal's own terms (J_kk = 0): real-times-complex sums in the inner loop
    cx<R> sx0[M], sy0[M], sx1[M], sy1[M];
#pragma unroll
    for (int k = 0; k < M; k++) sx0[k] = sy0[k] = sx1[k] = sy1[k] = cx<R>{R(0), R(0)};
    const R hs = R(0.5) * s;

    // ---- build S column by column (columns j in a loop; rows unrolled)
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        const cx<R> pj = pt.get(j), qj = pt.get(M + j);
        cx<R> Up, Uq, htf, htg;
        lc_U<M, R>(J, p, q, j, Up, Uq);
        lc_minus_ht_rows<R>(pj, qj, Up, Uq, gam, htf, htg);
        const cx<R> rf0 = two_rhs ? res.get(j) : htf;
        const cx<R> rg0 = two_rhs ? res.get(M + j) : htg;
        cx<R> ah, bh;
        R iv, sp, sq;
        g_frame_lc<R>(pj, qj, s, gomt, ah, bh, iv, sp, sq);
        // diagonal entries of gradient row j on (dwp_j, dwq_j):
        // (sp (-i t U_q + gamma (1-t) (p + q)) / 2, sq (i t U_p + gamma (1-t) (p + q)) / 2)
        const cx<R> gpq = cmul(gomt, cadd(pj, qj));
        const cx<R> Ajj = cscale(R(0.5) * sp, csub(gpq, cmul_i(cscale(s, Uq))));
        const cx<R> Bjj = cscale(R(0.5) * sq, cadd(gpq, cmul_i(cscale(s, Up))));
        const cx<R> q0 = cscale(iv, rg0), q1 = cscale(iv, htg);
        const cx<R> px0 = cmulc(ah, q0), py0 = cmulc(bh, q0);
        const cx<R> px1 = cmulc(ah, q1), py1 = cmulc(bh, q1);
        if (two_rhs && wr) out2.set(M + j, rg0);   // the residual's g row, for the recovery
        // the diagonal's own terms wait in row j of the right-hand-side columns (this
        // column's residual entries there were read above)
        A.set(j, M, csub(rf0, cadd(cmul(Ajj, px0), cmul(Bjj, py0))));
        if (two_rhs) A.set(j, M + 1, csub(htf, cadd(cmul(Ajj, px1), cmul(Bjj, py1))));
        // off-diagonal entries J_kj (q_k cb + p_k ca), with the factor i t / 2 and the scales
        // folded in (J_jj = 0 makes the k == j entry vanish; it is set below)
        const cx<R> cb = cmul_i(cscale(hs * sp, bh)), ca = cmul_i(cscale(hs * sq, ah));
        const cx<R> x0 = cscale(sp, px0), y0 = cscale(sq, py0);
        const cx<R> x1 = cscale(sp, px1), y1 = cscale(sq, py1);
#pragma unroll
        for (int k = 0; k < M; k++) {
            const R Jkj = J[k * NPHC_JSTRIDE + j];
            A.set(k, j, cscale(Jkj, cadd(cmul(q[k], cb), cmul(p[k], ca))));
            sx0[k] = cx<R>{fma(Jkj, x0.re, sx0[k].re), fma(Jkj, x0.im, sx0[k].im)};
            sy0[k] = cx<R>{fma(Jkj, y0.re, sy0[k].re), fma(Jkj, y0.im, sy0[k].im)};
            if (two_rhs) {
                sx1[k] = cx<R>{fma(Jkj, x1.re, sx1[k].re), fma(Jkj, x1.im, sx1[k].im)};
                sy1[k] = cx<R>{fma(Jkj, y1.re, sy1[k].re), fma(Jkj, y1.im, sy1[k].im)};
            }
        }
        A.set(j, j, csub(cmul(Ajj, bh), cmul(Bjj, ah)));
    }

    // right-hand sides into columns M and M + 1
#pragma unroll
    for (int k = 0; k < M; k++) {
        A.set(k, M, csub(A.get(k, M), cmul_i(cscale(hs, csub(cmul(q[k], sx0[k]), cmul(p[k], sy0[k]))))));
        if (two_rhs)
            A.set(k, M + 1, csub(A.get(k, M + 1), cmul_i(cscale(hs, csub(cmul(q[k], sx1[k]), cmul(p[k], sy1[k]))))));
    }

    bool ok = aug_lu_solve<M, R, BLOCK>(A, two_rhs, kest);

    // ---- back to (dp, dq) = (sp dwp, sq dwq),
    // (dwp, dwq) = conj(a^, b^) q_j + (b^, -a^) s_j
    R chk = R(0);
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        const cx<R> pj = pt.get(j), qj = pt.get(M + j);
        cx<R> ah, bh;
        R iv, sp, sq;
        g_frame_lc<R>(pj, qj, s, gomt, ah, bh, iv, sp, sq);
        const cx<R> htg = lc_minus_ht_g<R>(pj, qj, gam);
        const cx<R> q0 = cscale(iv, two_rhs ? out2.get(M + j) : htg);
        const cx<R> s0 = A.get(j, M);
        const cx<R> dp0 = cscale(sp, cadd(cmulc(ah, q0), cmul(bh, s0)));
        const cx<R> dq0 = cscale(sq, csub(cmulc(bh, q0), cmul(ah, s0)));
        chk += cabs2(dp0) + cabs2(dq0);
        if (two_rhs) {
            const cx<R> q1 = cscale(iv, htg);
            const cx<R> s1 = A.get(j, M + 1);
            const cx<R> dp1 = cscale(sp, cadd(cmulc(ah, q1), cmul(bh, s1)));
            const cx<R> dq1 = cscale(sq, csub(cmulc(bh, q1), cmul(ah, s1)));
            chk += cabs2(dp1) + cabs2(dq1);
            if (wr) {
                out2.set(j, dp1);
                out2.set(M + j, dq1);
            }
        }
        if (wr) {
            out1.set(j, dp0);
            out1.set(M + j, dq0);
        }
    }
    return ok && finite_r(chk);
}

// -H(z, t) at the light-cone point in `pt`, evaluated with compensated sums (float-float
// for FP32, double-double for FP64) and exact products, then rounded once: the error is
// ~u^2 of the terms instead of u, so a Newton corrector driven by it converges to the
// rounding of the path point even when H_z is far from well conditioned (mixed-precision
// iterative refinement; at large ||z|| the terms of H are ~||z||^2 while H itself is near
// zero).  The coefficients J, gamma (1-t) and t enter as their values in R; every other
// factor is a product of two coordinates (or one coordinate and a power of two).
template <int M, class R, int BLOCK>
__device__ __forceinline__ void xy_residual_comp(const R *__restrict__ J,
                                                 const SVec<R, BLOCK> &pt, R s, R omt,
                                                 cx<R> gam, const SVec<R, BLOCK> &out, bool wr) {
    using E = EFT<R>;
    const cx<R> gomt = cx<R>{E::mul(omt, gam.re), E::mul(omt, gam.im)};
    cx<R> p[M], q[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        p[k] = pt.get(k);
        q[k] = pt.get(M + k);
    }
    const ext<R> zero = {R(0), R(0)};
    const R hs = R(0.5) * s;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const cx<R> pk = pt.get(k), qk = pt.get(M + k);
        const R *Jk = J + k * NPHC_JSTRIDE;
        ext<R> upr = {Jk[M], R(0)}, upi = zero, uqr = {Jk[M], R(0)}, uqi = zero;
#pragma unroll
        for (int l = 0; l < M; l++) {   // J_kk = 0 adds exact zeros
            const R Jl = Jk[l];
            ext_acc(upr, Jl, p[l].re);
            ext_acc(upi, Jl, p[l].im);
            ext_acc(uqr, Jl, q[l].re);
            ext_acc(uqi, Jl, q[l].im);
        }
        // D = q U_p - p U_q, f = i D / 2
        ext<R> dr = zero, di = zero;
        ext_acc_ext(dr, qk.re, upr);
        ext_acc_ext(dr, -qk.im, upi);
        ext_acc_ext(dr, -pk.re, uqr);
        ext_acc_ext(dr, pk.im, uqi);
        ext_acc_ext(di, qk.re, upi);
        ext_acc_ext(di, qk.im, upr);
        ext_acc_ext(di, -pk.re, uqi);
        ext_acc_ext(di, -pk.im, uqr);
        // X = x^2 - 1 = (p^2 + 2 p q + q^2) / 4 - 1, Y = y^2 - 1 = -(p^2 - 2 p q + q^2) / 4 - 1,
        // G = p q - 1, as two-word numbers (the factors 1/4, 1/2 are exact)
        ext<R> xr = {R(-1), R(0)}, xi = zero, yr = {R(-1), R(0)}, yi = zero;
        ext<R> gr = {R(-1), R(0)}, gi = zero;
        ext_acc(xr, R(0.25) * pk.re, pk.re);
        ext_acc(xr, R(-0.25) * pk.im, pk.im);
        ext_acc(xr, R(0.5) * pk.re, qk.re);
        ext_acc(xr, R(-0.5) * pk.im, qk.im);
        ext_acc(xr, R(0.25) * qk.re, qk.re);
        ext_acc(xr, R(-0.25) * qk.im, qk.im);
        ext_acc(xi, R(0.5) * pk.re, pk.im);
        ext_acc(xi, R(0.5) * pk.re, qk.im);
        ext_acc(xi, R(0.5) * pk.im, qk.re);
        ext_acc(xi, R(0.5) * qk.re, qk.im);
        ext_acc(yr, R(-0.25) * pk.re, pk.re);
        ext_acc(yr, R(0.25) * pk.im, pk.im);
        ext_acc(yr, R(0.5) * pk.re, qk.re);
        ext_acc(yr, R(-0.5) * pk.im, qk.im);
        ext_acc(yr, R(-0.25) * qk.re, qk.re);
        ext_acc(yr, R(0.25) * qk.im, qk.im);
        ext_acc(yi, R(-0.5) * pk.re, pk.im);
        ext_acc(yi, R(0.5) * pk.re, qk.im);
        ext_acc(yi, R(0.5) * pk.im, qk.re);
        ext_acc(yi, R(-0.5) * qk.re, qk.im);
        ext_acc(gr, pk.re, qk.re);
        ext_acc(gr, -pk.im, qk.im);
        ext_acc(gi, pk.re, qk.im);
        ext_acc(gi, pk.im, qk.re);
        // H_f = gomt X + t f ;  H_g = gomt Y + t G
        ext<R> hfr = zero, hfi = zero, hgr = zero, hgi = zero;
        ext_acc_ext(hfr, gomt.re, xr);
        ext_acc_ext(hfr, -gomt.im, xi);
        ext_acc_ext(hfr, -hs, di);
        ext_acc_ext(hfi, gomt.re, xi);
        ext_acc_ext(hfi, gomt.im, xr);
        ext_acc_ext(hfi, hs, dr);
        ext_acc_ext(hgr, gomt.re, yr);
        ext_acc_ext(hgr, -gomt.im, yi);
        ext_acc_ext(hgr, s, gr);
        ext_acc_ext(hgi, gomt.re, yi);
        ext_acc_ext(hgi, gomt.im, yr);
        ext_acc_ext(hgi, s, gi);
        if (wr) {
            out.set(k, cx<R>{-ext_val(hfr), -ext_val(hfi)});
            out.set(M + k, cx<R>{-ext_val(hgr), -ext_val(hgi)});
        }
    }
}
