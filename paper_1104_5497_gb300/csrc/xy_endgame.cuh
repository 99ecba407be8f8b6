// xy_endgame.cuh -- FP64 work at t = 1 on the endpoints of the XY ring:
//   refinement: Newton's method on P to full double precision (section "Numerical
//     Polynomial Homotopy Continuation Method" refines every endpoint to machine
//     precision before certifying it), with P evaluated by exact products and
//     double-double sums (eg_minus_p);
//   the solution tolerance Delta_sol on ||P(z)||_inf;
//   alpha-theory certification (the alphaCertified step of the same section):
//     beta = ||DP^-1 P||_2, gamma <= ||DP^-1||_F ||D^2 P / 2|| (P is quadratic, so
//     D^k P = 0 for k >= 3 and Smale's gamma is ||DP^-1 D^2P/2|| exactly), certified when
//     alpha = beta gamma < (13 - 3 sqrt 17) / 4; real when z and Re z share their zero
//     (alpha < 0.03 and ||Im z|| < 1 / (20 gamma)) and the test passes at Re z (a real
//     point of a real system: Newton's iterates stay real), otherwise non-real when
//     ||z - conj z|| > 2 (beta(z) + beta(conj z)), i.e. ||Im z|| > 2 beta, else undecided;
//   classification of real stationary points (introduction and section "A First
//     Application"): theta_k = atan2(s_k, c_k) in (-pi, pi], the Hessian of
//     V = sum_{i<j} J_ij (1 - cos(theta_i - theta_j)) in theta_1..theta_M, its number of
//     negative eigenvalues (cyclic Jacobi), and V.
//
// Linear algebra at t = 1 (the structure of xy_solve.cuh): in the unitary per-site frame
// W, (dx_j, dy_j) = conj(a^_j, b^_j) q_j + (b^_j, -a^_j) s_j, the Jacobian becomes
//   DP W = [[C, S], [D, 0]],   D = diag(nu_j), nu_j = |(a_j, b_j)| = 1 / iv_j,
//   C_kj = A_kj conj(a^_j) + B_kj conj(b^_j),  S_kj = A_kj b^_j - B_kj a^_j,
// (A, B: derivatives of the gradient rows in c and s) with inverse
//   [[0, D^-1], [S^-1, -S^-1 C D^-1]],
// so a solve costs one M x M system, and, W being unitary,
//   ||DP^-1||_F^2 = sum_j iv_j^2 + ||S^-1||_F^2 + ||S^-1 C D^-1||_F^2
// needs only 2M triangular solves after one Householder QR of S (stored: R above the
// diagonal with a real diagonal, the reflectors below, conj(tau) aside).
//
// The refinement certifies the iterate whose Newton correction met the tolerance, from
// the factorisation of that iteration, and outputs its Newton iterate.
//
// Storage: one endpoint per thread, interleaved across the 32 threads of a block
// (element i of a thread's array at [i * 32 + lane]) so that the rolled loops index it
// at run time without local memory: the per-site arrays, point and vectors in shared
// memory, the M x M factor in shared memory too or, when a solve provides a scratch
// buffer, in global memory (L2-resident), which leaves room for more warps per SM.
#pragma once

#include "nphc_internal.cuh"

#define EG_BLOCK 32

// The certification threshold: half of Smale's (13 - 3 sqrt 17) / 4.  alphaCertified
// decides in exact arithmetic; an FP64 test keeps a factor of two so that rounding cannot
// carry a point near a singular solution set across the constant (on the N = 4 ring a
// point of the positive-dimensional family reached alpha = 0.115 < 0.158).
#define NPHC_ALPHA_CERT (0.5 * (13.0 - 3.0 * sqrt(17.0)) / 4.0)


// One thread's array of complex doubles in shared memory.
struct EGVec {
    cx<double> *p;
    __device__ __forceinline__ cx<double> get(int i) const { return p[i * EG_BLOCK]; }
    __device__ __forceinline__ void set(int i, cx<double> v) const { p[i * EG_BLOCK] = v; }
};

// Per-thread working set of the endgame (complex doubles, in this order).  The M x M
// matrix S comes last: in shared memory with the rest, or (refinement launches given a
// scratch buffer) in global memory, interleaved across the launch's threads, so that the
// shared part alone sets the occupancy.
template <int M>
struct EGLayout {
    static constexpr int TQ = 0;                // conj(tau) of the reflectors
    static constexpr int AH = TQ + M;           // frame a^
    static constexpr int BH = AH + M;           // frame b^
    static constexpr int IV = BH + M;           // iv (real part)
    static constexpr int AD = IV + M;           // d f_j / d c_j
    static constexpr int BD = AD + M;           // d f_j / d s_j
    static constexpr int X = BD + M;            // c_1..c_M
    static constexpr int Y = X + M;             // s_1..s_M
    static constexpr int R = Y + M;             // right-hand side / residual, 2M
    static constexpr int D = R + 2 * M;         // solution, 2M
    static constexpr int S = D + 2 * M;         // M x M, column-major: entry (i, c) at c M + i
    static constexpr int TOTAL = S + M * M;
};

// Shared memory per thread, with S or without it (S in a global scratch buffer).
template <int M>
constexpr size_t eg_smem_per_thread(bool with_s = true) {
    return sizeof(cx<double>) * (size_t)(with_s ? EGLayout<M>::TOTAL : EGLayout<M>::S);
}

template <int M>
struct EG {
    cx<double> *base;   // this thread's first entry in shared memory (stride EG_BLOCK)
    cx<double> *sp;     // this thread's entry (0, 0) of S, in shared or global memory
    int64_t ss;         // S's stride between entries
    __device__ __forceinline__ EGVec v(int off) const { return EGVec{base + off * EG_BLOCK}; }
    __device__ __forceinline__ cx<double> S(int i, int c) const { return sp[(c * M + i) * ss]; }
    __device__ __forceinline__ void setS(int i, int c, cx<double> a) const { sp[(c * M + i) * ss] = a; }
};

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

// -P(z) into R, with exact products and double-double sums; returns ||P||_inf.
template <int M>
__device__ double eg_minus_p(const EG<M> &G, const double *__restrict__ J) {
    const EGVec X = G.v(EGLayout<M>::X), Y = G.v(EGLayout<M>::Y), R = G.v(EGLayout<M>::R);
    double res = 0.0;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const double *Jk = J + k * NPHC_JSTRIDE;
        dd ur = {Jk[M], 0.0}, ui = {0.0, 0.0}, wr = {0.0, 0.0}, wi = {0.0, 0.0};
#pragma unroll 1
        for (int l = 0; l < M; l++) {   // J_kk = 0 adds exact zeros
            const cx<double> xl = X.get(l), yl = Y.get(l);
            ur = dd_add(ur, dd_two_prod(Jk[l], xl.re));
            ui = dd_add(ui, dd_two_prod(Jk[l], xl.im));
            wr = dd_add(wr, dd_two_prod(Jk[l], yl.re));
            wi = dd_add(wi, dd_two_prod(Jk[l], yl.im));
        }
        const cx<double> xk = X.get(k), yk = Y.get(k);
        // f = y u - x w
        const dd fr = dd_add(dd_add(dd_mul_d(ur, yk.re), dd_mul_d(ui, -yk.im)),
                             dd_add(dd_mul_d(wr, -xk.re), dd_mul_d(wi, xk.im)));
        const dd fi = dd_add(dd_add(dd_mul_d(ui, yk.re), dd_mul_d(ur, yk.im)),
                             dd_add(dd_mul_d(wi, -xk.re), dd_mul_d(wr, -xk.im)));
        // g = c^2 + s^2 - 1
        dd gr = dd_add(dd_add(dd_two_prod(xk.re, xk.re), dd_two_prod(-xk.im, xk.im)),
                       dd_add(dd_two_prod(yk.re, yk.re), dd_two_prod(-yk.im, yk.im)));
        gr = dd_add(gr, dd{-1.0, 0.0});
        const dd gi = dd_add(dd_two_prod(2.0 * xk.re, xk.im), dd_two_prod(2.0 * yk.re, yk.im));
        const cx<double> f = cx<double>{dd_val(fr), dd_val(fi)};
        const cx<double> g = cx<double>{dd_val(gr), dd_val(gi)};
        res = fmax(res, fmax(sqrt(cabs2(f)), sqrt(cabs2(g))));
        R.set(k, cx<double>{-f.re, -f.im});
        R.set(M + k, cx<double>{-g.re, -g.im});
    }
    return res;
}

// Householder QR of the M x M matrix G.S in place: R above the diagonal with a real
// diagonal (stored as (beta, 0)), the reflectors (1, v) below it, conj(tau) in TQ.
// Returns false when the matrix is singular.
template <int M>
__device__ bool eg_qr(const EG<M> &G) {
    const EGVec TQ = G.v(EGLayout<M>::TQ);
    bool ok = true;
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        const cx<double> al = G.S(k, k);
        double xn2 = 0.0;
#pragma unroll 1
        for (int i = k + 1; i < M; i++) xn2 += cabs2(G.S(i, k));
        const double an = sqrt(cabs2(al) + xn2);
        ok = ok && an > 0.0;
        const double beta = al.re >= 0.0 ? -an : an;
        const cx<double> tauc = cx<double>{(beta - al.re) / beta, al.im / beta};
        const cx<double> sc = crecip(cx<double>{al.re - beta, al.im});
#pragma unroll 1
        for (int i = k + 1; i < M; i++) G.setS(i, k, cmul(G.S(i, k), sc));
        G.setS(k, k, cx<double>{beta, 0.0});
        TQ.set(k, tauc);
#pragma unroll 1
        for (int c = k + 1; c < M; c++) {
            cx<double> wv = G.S(k, c);
#pragma unroll 1
            for (int i = k + 1; i < M; i++) wv = cadd(wv, cmulc(G.S(i, k), G.S(i, c)));
            wv = cmul(tauc, wv);
            G.setS(k, c, csub(G.S(k, c), wv));
#pragma unroll 1
            for (int i = k + 1; i < M; i++) G.setS(i, c, csub(G.S(i, c), cmul(G.S(i, k), wv)));
        }
    }
    return ok;
}

// Frames, diagonal Jacobian entries and the Householder QR of S at the point (X, Y).
// Returns false when S is singular.
template <int M>
__device__ bool eg_factor(const EG<M> &G, const double *__restrict__ J) {
    using L = EGLayout<M>;
    const EGVec X = G.v(L::X), Y = G.v(L::Y), AH = G.v(L::AH), BH = G.v(L::BH), IV = G.v(L::IV),
                AD = G.v(L::AD), BD = G.v(L::BD);
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        const double *Jj = J + j * NPHC_JSTRIDE;
        cx<double> u = cx<double>{Jj[M], 0.0}, w = cx<double>{0.0, 0.0};
#pragma unroll 1
        for (int l = 0; l < M; l++) {
            const cx<double> xl = X.get(l), yl = Y.get(l);
            u.re += Jj[l] * xl.re;
            u.im += Jj[l] * xl.im;
            w.re += Jj[l] * yl.re;
            w.im += Jj[l] * yl.im;
        }
        AD.set(j, cx<double>{-w.re, -w.im});
        BD.set(j, u);
        const cx<double> a = cscale(2.0, X.get(j)), b = cscale(2.0, Y.get(j));
        const double iv = rsqrt(cabs2(a) + cabs2(b));
        IV.set(j, cx<double>{iv, 0.0});
        AH.set(j, cscale(iv, a));
        BH.set(j, cscale(iv, b));
    }
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        const cx<double> ah = AH.get(j), bh = BH.get(j);
#pragma unroll 1
        for (int k = 0; k < M; k++) {
            cx<double> e;
            if (k == j)
                e = csub(cmul(AD.get(j), bh), cmul(BD.get(j), ah));
            else
                e = cscale(J[k * NPHC_JSTRIDE + j], cadd(cmul(Y.get(k), bh), cmul(X.get(k), ah)));
            G.setS(k, j, e);
        }
    }
    return eg_qr<M>(G);
}

// b <- R^-1 Q^H b (b: M entries of a per-thread array); returns ||b||^2 afterwards.
template <int M>
__device__ double eg_schur_solve(const EG<M> &G, const EGVec &b) {
    const EGVec TQ = G.v(EGLayout<M>::TQ);
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        cx<double> wv = b.get(k);
#pragma unroll 1
        for (int i = k + 1; i < M; i++) wv = cadd(wv, cmulc(G.S(i, k), b.get(i)));
        wv = cmul(TQ.get(k), wv);
        b.set(k, csub(b.get(k), wv));
#pragma unroll 1
        for (int i = k + 1; i < M; i++) b.set(i, csub(b.get(i), cmul(G.S(i, k), wv)));
    }
    double n2 = 0.0;
#pragma unroll 1
    for (int k = M - 1; k >= 0; k--) {
        cx<double> acc = b.get(k);
#pragma unroll 1
        for (int c = k + 1; c < M; c++) acc = csub(acc, cmul(G.S(k, c), b.get(c)));
        acc = cscale(1.0 / G.S(k, k).re, acc);
        b.set(k, acc);
        n2 += cabs2(acc);
    }
    return n2;
}

// C_kj (the q_j-coefficient of gradient row k in the frame).
template <int M>
__device__ __forceinline__ cx<double> eg_C(const EG<M> &G, const double *__restrict__ J, int k,
                                           int j) {
    using L = EGLayout<M>;
    const cx<double> ah = G.v(L::AH).get(j), bh = G.v(L::BH).get(j);
    if (k == j)
        return cadd(cmulc(ah, G.v(L::AD).get(j)), cmulc(bh, G.v(L::BD).get(j)));
    const double Jkj = J[k * NPHC_JSTRIDE + j];
    return cscale(Jkj, csub(cmulc(ah, G.v(L::Y).get(k)), cmulc(bh, G.v(L::X).get(k))));
}

// D <- DP^-1 R (after eg_factor); returns ||D||^2.
template <int M>
__device__ double eg_solve(const EG<M> &G, const double *__restrict__ J) {
    using L = EGLayout<M>;
    const EGVec R = G.v(L::R), Dv = G.v(L::D), IV = G.v(L::IV), AH = G.v(L::AH), BH = G.v(L::BH);
    // q_j = iv_j r_gj into D[M + j]; Schur right-hand side r_fk - sum_j C_kj q_j into D[k]
#pragma unroll 1
    for (int j = 0; j < M; j++) Dv.set(M + j, cscale(IV.get(j).re, R.get(M + j)));
#pragma unroll 1
    for (int k = 0; k < M; k++) {
        cx<double> acc = R.get(k);
#pragma unroll 1
        for (int j = 0; j < M; j++) acc = csub(acc, cmul(eg_C<M>(G, J, k, j), Dv.get(M + j)));
        Dv.set(k, acc);
    }
    eg_schur_solve<M>(G, Dv);
    double n2 = 0.0;
#pragma unroll 1
    for (int j = 0; j < M; j++) {
        const cx<double> ah = AH.get(j), bh = BH.get(j), q = Dv.get(M + j), sj = Dv.get(j);
        const cx<double> dx = cadd(cmulc(ah, q), cmul(bh, sj));
        const cx<double> dy = csub(cmulc(bh, q), cmul(ah, sj));
        Dv.set(j, dx);
        Dv.set(M + j, dy);
        n2 += cabs2(dx) + cabs2(dy);
    }
    return n2;
}

// ||DP^-1||_F after eg_factor (block formula above); uses D as scratch.
template <int M>
__device__ double eg_inv_fro(const EG<M> &G, const double *__restrict__ J) {
    using L = EGLayout<M>;
    const EGVec Dv = G.v(L::D), IV = G.v(L::IV);
    double s = 0.0;
#pragma unroll 1
    for (int j = 0; j < M; j++) s += IV.get(j).re * IV.get(j).re;
    // columns of S^-1 and of S^-1 C D^-1
#pragma unroll 1
    for (int col = 0; col < 2 * M; col++) {
        const int j = col < M ? col : col - M;
#pragma unroll 1
        for (int k = 0; k < M; k++)
            Dv.set(k, col < M ? cx<double>{k == j ? 1.0 : 0.0, 0.0}
                              : cscale(IV.get(j).re, eg_C<M>(G, J, k, j)));
        s += eg_schur_solve<M>(G, Dv);
    }
    return sqrt(s);
}

// shortcut = 1: entries handed off by the FP32 pass close to t = 1 are refined at t = 1
// directly (Newton on P from the hand-off point: for a path to a nonsingular solution xi,
// z(t) = xi + (1 - t) z'(1) + ..., so the point is already in xi's Newton basin).  The
// first Newton correction must stay below SHORTCUT_TRUST (1 + ||z||); an entry that
// certifies becomes NPHC_PATH_REACHED, any other entry is left untouched.
#define SHORTCUT_TRUST 1e-2

// The system an endgame kernel works on, as a policy for refine_body: the unknowns
// (NZ, stored in G's X then Y), -P into R, the factorisation of DP, the Newton step
// D = DP^-1 R, ||DP^-1||_F and ||D^2 P / 2||.  EGXY: the XY ring (frames + Schur QR).
template <int M>
struct EGXY {
    using Sys = XYSys;
    static constexpr int DIM = M;        // EG<DIM> storage
    static constexpr int NZ = 2 * M;
    static __device__ __forceinline__ cx<double> zget(const EG<M> &G, int k) {
        return k < M ? G.v(EGLayout<M>::X).get(k) : G.v(EGLayout<M>::Y).get(k - M);
    }
    static __device__ __forceinline__ void zset(const EG<M> &G, int k, cx<double> v) {
        if (k < M) G.v(EGLayout<M>::X).set(k, v);
        else G.v(EGLayout<M>::Y).set(k - M, v);
    }
    static __device__ __forceinline__ double minus_p(const EG<M> &G, const Sys &S) {
        return eg_minus_p<M>(G, S.Jd);
    }
    static __device__ __forceinline__ bool factor(const EG<M> &G, const Sys &S) {
        return eg_factor<M>(G, S.Jd);
    }
    static __device__ __forceinline__ double solve(const EG<M> &G, const Sys &S) {
        return eg_solve<M>(G, S.Jd);
    }
    static __device__ __forceinline__ double inv_fro(const EG<M> &G, const Sys &S) {
        return eg_inv_fro<M>(G, S.Jd);
    }
    // ||DP||_F after factor: gradient row k has J_kj y_k, -J_kj x_k (free j != k), -w_k,
    // u_k; constraint row k has 2 x_k, 2 y_k
    static __device__ __forceinline__ double jac_fro(const EG<M> &G, const Sys &S) {
        using L = EGLayout<M>;
        double f = 0.0;
#pragma unroll 1
        for (int k = 0; k < M; k++) {
            const double xy = cabs2(G.v(L::X).get(k)) + cabs2(G.v(L::Y).get(k));
            double jj = 0.0;
#pragma unroll 1
            for (int j = 0; j < M; j++) jj += S.Jd[k * NPHC_JSTRIDE + j] * S.Jd[k * NPHC_JSTRIDE + j];
            f += jj * xy + cabs2(G.v(L::AD).get(k)) + cabs2(G.v(L::BD).get(k)) + 4.0 * xy;
        }
        return sqrt(f);
    }
    static __device__ __forceinline__ double d2norm(const Sys &S) { return S.d2norm; }
};

// beta = ||DP^-1 P||, ||DP^-1||_F and ||P||_inf at the point in G.  False if singular:
// at a point of a positive-dimensional solution set P vanishes to double-double precision
// (beta is tiny) while rounding leaves the computed DP^-1 merely huge, and the soft alpha
// test alone can pass there, so a Frobenius condition number ||DP||_F ||DP^-1||_F above
// kappa_sing max(1, ||z||_inf^2) counts as singular.  The bound grows with ||z||_inf^2 like
// the solution tolerance: the equations are quadratic, the Jacobian's entries grow like
// ||z|| and an isolated solution near the solution set at infinity has a smallest singular
// value shrinking like 1 / ||z|| (a solution of norm 1e6 has a condition number ~1e12).
// The same from a factorisation already made at the point in G: fro = ||DP||_F, dn =
// ||DP^-1 P|| from its solve (inv_fro takes D as scratch).
template <class Q>
__device__ bool eg_certify_factored(const EG<Q::DIM> &G, const typename Q::Sys &S, double fro,
                                    double dn, double &beta, double &invF) {
    beta = dn;
    invF = Q::inv_fro(G, S);
    double zi = 0.0;
#pragma unroll 1
    for (int k = 0; k < Q::NZ; k++) zi = fmax(zi, sqrt(cabs2(Q::zget(G, k))));
    return isfinite(beta) && isfinite(invF) && fro * invF <= S.kappa_sing * fmax(1.0, zi * zi);
}

template <class Q>
__device__ bool eg_beta_invnorm_p(const EG<Q::DIM> &G, const typename Q::Sys &S, double &beta,
                                  double &invF, double &res) {
    res = Q::minus_p(G, S);
    if (!Q::factor(G, S)) return false;
    const double fro = Q::jac_fro(G, S);
    const double dn = sqrt(Q::solve(G, S));
    return eg_certify_factored<Q>(G, S, fro, dn, beta, invF);
}

// Refinement and certification of entry e.  Returns true when e still needs the
// alpha-test at Re z (its refined z is already written out; the caller runs the test).
template <class Q>
__device__ bool eg_refine_certify_one(const EG<Q::DIM> &G, const typename Q::Sys &S,
                                      double tol_sol, double refine_eps, int refine_iters,
                                      const EPView &ep, int64_t e, int shortcut) {
    constexpr int NZ = Q::NZ;
    const EGVec Dv = G.v(EGLayout<Q::DIM>::D);
    const int64_t cnt = ep.count;
    const double alpha0 = NPHC_ALPHA_CERT;
    const int st = ep.status[e];
    const bool sc = shortcut && (st == NPHC_PATH_HANDOFF || st == NPHC_PATH_HANDOFF_COND);
    if (!sc) {
        ep.alpha[e] = INFINITY;
        ep.beta[e] = INFINITY;
        ep.gamma[e] = INFINITY;
        ep.resid[e] = INFINITY;
        if (st == NPHC_PATH_DIVERGED) {
            ep.cls[e] = NPHC_END_NONE;
            return false;
        }
        if (st != NPHC_PATH_REACHED) {
            ep.cls[e] = NPHC_END_FAILED;
            return false;
        }
    }
#pragma unroll 1
    for (int k = 0; k < NZ; k++) Q::zset(G, k, cx<double>{ep.z_re[k * cnt + e], ep.z_im[k * cnt + e]});
    int cls = NPHC_END_SINGULAR;
    bool finite = true;
    double beta = INFINITY, invF = INFINITY, res = INFINITY;
    bool certified = false, cert_ok = false;
    // Newton refinement on P.  The iteration whose correction meets refine_eps certifies its
    // own point z_k from the factorisation it has just made (beta = ||dz_k||, exactly what a
    // separate certification at z_k computes), and the output is z_k's Newton iterate
    // z_k + dz_k, closer still to the same zero: one evaluation, factorisation and solve
    // less than certifying the output point afresh
#pragma unroll 1
    for (int it = 0; it < refine_iters; it++) {
        const double rk = Q::minus_p(G, S);
        if (!Q::factor(G, S)) break;
        const double dn = sqrt(Q::solve(G, S));
        double z2 = 0.0;
#pragma unroll 1
        for (int k = 0; k < NZ; k++) z2 += cabs2(Q::zget(G, k));
        if (sc && it == 0 && !(dn <= SHORTCUT_TRUST * (1.0 + sqrt(z2)))) return false;   // not in a basin
        if (!isfinite(dn) || !isfinite(z2)) {
            finite = false;
            break;
        }
        const bool last = dn <= refine_eps * (1.0 + sqrt(z2));
        const EGVec Step = last ? G.v(EGLayout<Q::DIM>::R) : Dv;
        if (last) {
#pragma unroll 1
            for (int k = 0; k < NZ; k++) Step.set(k, Dv.get(k));   // inv_fro takes D as scratch
            const double fro = Q::jac_fro(G, S);
            cert_ok = eg_certify_factored<Q>(G, S, fro, dn, beta, invF);
            res = rk;
            certified = true;
        }
        double zn = 0.0;
#pragma unroll 1
        for (int k = 0; k < NZ; k++) {
            const cx<double> zk = cadd(Q::zget(G, k), Step.get(k));
            Q::zset(G, k, zk);
            zn += cabs2(zk);
        }
        if (!isfinite(zn)) {
            finite = false;
            break;
        }
        if (last) break;
    }
    if (finite && !certified) cert_ok = eg_beta_invnorm_p<Q>(G, S, beta, invF, res);
    double alpha = INFINITY, gam = INFINITY;
    bool real_test = false;
    if (finite && cert_ok) {
        gam = invF * Q::d2norm(S);
        alpha = beta * gam;
        // Delta_sol relative to the size of the (quadratic) terms: max(1, ||z||_inf^2)
        double zi = 0.0, im2 = 0.0;
#pragma unroll 1
        for (int k = 0; k < NZ; k++) {
            const cx<double> zk = Q::zget(G, k);
            zi = fmax(zi, sqrt(cabs2(zk)));
            im2 += zk.im * zk.im;
        }
        if (res <= tol_sol * fmax(1.0, zi * zi) && alpha < alpha0) {
            // z and Re z share their associated zero when alpha < 0.03 and
            // ||Im z|| < 1 / (20 gamma): then the real test at Re z decides (queued)
            const double im = sqrt(im2);
            if (alpha < 0.03 && im < 1.0 / (20.0 * gam))
                real_test = true;
            else
                cls = im > 2.0 * beta ? NPHC_END_NONREAL : NPHC_END_UNDECIDED;
        }
    } else {
        beta = INFINITY;
    }
    if (sc && !(real_test || cls == NPHC_END_NONREAL || cls == NPHC_END_UNDECIDED))
        return false;   // left for FP64 tracking
    ep.alpha[e] = alpha;
    ep.beta[e] = beta;
    ep.gamma[e] = gam;
    ep.resid[e] = finite ? res : INFINITY;
    if (sc) {
        ep.status[e] = NPHC_PATH_REACHED;
        ep.t[e] = 1.0;
    }
#pragma unroll 1
    for (int k = 0; k < NZ; k++) {
        const cx<double> zk = Q::zget(G, k);
        ep.z_re[k * cnt + e] = zk.re;
        ep.z_im[k * cnt + e] = zk.im;
    }
    if (!real_test) ep.cls[e] = cls;
    return real_test;
}

// The alpha-test at Re z of a certified entry e that shares its zero with Re z: real
// when it passes there; otherwise non-real when ||Im z|| > 2 beta (z and conj z then
// have distinct zeros), else undecided.
template <class Q>
__device__ void eg_real_test(const EG<Q::DIM> &G, const typename Q::Sys &S, const EPView &ep,
                             int64_t e) {
    const int64_t cnt = ep.count;
    const double alpha0 = NPHC_ALPHA_CERT;
    double im2 = 0.0;
#pragma unroll 1
    for (int k = 0; k < Q::NZ; k++) {
        const double yi = ep.z_im[k * cnt + e];
        im2 += yi * yi;
        Q::zset(G, k, cx<double>{ep.z_re[k * cnt + e], 0.0});
    }
    double br, ir, rr;
    if (eg_beta_invnorm_p<Q>(G, S, br, ir, rr) && br * ir * Q::d2norm(S) < alpha0)
        ep.cls[e] = NPHC_END_REAL;
    else
        ep.cls[e] = sqrt(im2) > 2.0 * ep.beta[e] ? NPHC_END_NONREAL : NPHC_END_UNDECIDED;
}

// One warp per block.  Entries are taken 32 at a time; the few that need the real test
// (about one in thirty at N = 10) go to a per-warp queue that is drained 32 at a time,
// so that the test runs on full warps instead of costing most warps a pass with one
// active lane.  With wl.state set (a scratch buffer of at least gridDim.x x EG_BLOCK
// threads' matrices), S lives there: the launch then needs shared memory for the rest
// only, and fits more warps per SM (GB300's FP64 pipes are per SM sub-partition: at M = 9
// four warps use all four where the 3 KB per thread of the whole set allowed two).
template <class Q>
__device__ __forceinline__ void refine_body(const typename Q::Sys &S, double tol_sol,
                                            double refine_eps, int refine_iters, const EPView &ep,
                                            const WorkList &wl, int shortcut) {
    using L = EGLayout<Q::DIM>;
    extern __shared__ __align__(16) unsigned char egraw[];
    __shared__ int64_t rq[2 * EG_BLOCK];
    const int lane = threadIdx.x;
    cx<double> *const sb = reinterpret_cast<cx<double> *>(egraw) + lane;
    const EG<Q::DIM> G = wl.state
        ? EG<Q::DIM>{sb, reinterpret_cast<cx<double> *>(wl.state) + (int64_t)blockIdx.x * EG_BLOCK + lane,
                     (int64_t)gridDim.x * EG_BLOCK}
        : EG<Q::DIM>{sb, sb + L::S * EG_BLOCK, EG_BLOCK};
    const int64_t total = worklist_size(wl, ep.count);
    int qn = 0;   // queued real tests (the same in every lane)
    for (int64_t base = (int64_t)blockIdx.x * EG_BLOCK; base < total;
         base += (int64_t)gridDim.x * EG_BLOCK) {
        const int64_t i = base + lane;
        int64_t e = -1;
        bool rt = false;
        if (i < total) e = worklist_entry(wl, i, ep.count);   // -1: rejected (debug)
        if (e >= 0)
            rt = eg_refine_certify_one<Q>(G, S, tol_sol, refine_eps, refine_iters, ep, e, shortcut);
        const unsigned m = __ballot_sync(0xffffffffu, rt);
        if (rt) rq[qn + __popc(m & ((1u << lane) - 1u))] = e;
        qn += __popc(m);
        __syncwarp();
        if (qn >= EG_BLOCK) {
            eg_real_test<Q>(G, S, ep, rq[qn - EG_BLOCK + lane]);
            qn -= EG_BLOCK;
            __syncwarp();
        }
    }
    if (lane < qn) eg_real_test<Q>(G, S, ep, rq[lane]);
}

template <int M>
__global__ void __launch_bounds__(EG_BLOCK)
    xy_refine_certify_kernel(const __grid_constant__ XYSys S, double tol_sol, double refine_eps,
                             int refine_iters, const EPView ep, const WorkList wl, int shortcut) {
    refine_body<EGXY<M>>(S, tol_sol, refine_eps, refine_iters, ep, wl, shortcut);
}

template <int M>
__global__ void __launch_bounds__(128)
    xy_classify_kernel(const __grid_constant__ XYSys S, const EPView ep, double *theta,
                       int32_t *index, double *energy, double *min_eig, double *log_abs_det,
                       const int32_t *list, const int32_t *list_count) {
    // every entry, or the listed ones: the real stationary points packed 32 to a warp, so
    // that the FP64 Jacobi runs on full warps (GB300's FP64 pipe charges a warp instruction
    // whatever the number of active lanes, and scattered real points cost a warp each)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = ep.count;
    int64_t e = i;
    if (list) {
        if (i >= *list_count) return;
        e = list[i];
        if (!NPHC_VALID(e >= 0 && e < cnt, 5)) return;
    }
    if (e >= cnt) return;
    if (ep.cls[e] != NPHC_END_REAL) {
        index[e] = -1;
        energy[e] = 0.0;
        if (min_eig) min_eig[e] = 0.0;
        if (log_abs_det) log_abs_det[e] = 0.0;
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
    double mn = INFINITY, ld = 0.0;
    for (int k = 0; k < M; k++) {
        const double w = H[k * M + k];
        if (w < 0.0) neg++;
        mn = fmin(mn, fabs(w));
        ld += log(fabs(w));   // log |det H| = sum of log |eigenvalue|
    }
    index[e] = neg;
    energy[e] = V;
    if (min_eig) min_eig[e] = mn;
    if (log_abs_det) log_abs_det[e] = ld;
}

// Gradient with respect to the couplings of a loss L(V*, theta*) summed over real
// stationary points (not part of the paper's method: derivatives of its outputs).  At
// theta* the gradient G = grad_theta V vanishes, so dV*/dJ_ij = 1 - cos(theta_i - theta_j)
// (envelope), and d theta*/dJ_ij = -H^-1 dG/dJ_ij (implicit function theorem); with
// H lambda = dL/dtheta (lambda_N = 0) and dG_i/dJ_ij = sin(theta_i - theta_j) = -dG_j/dJ_ij:
//   dL/dJ_ij = gV (1 - cos(theta_i - theta_j)) - (lambda_i - lambda_j) sin(theta_i - theta_j).
// One stationary point per thread (theta: [count * M] row per point; g_energy [count] and
// g_theta [count * M] may be NULL), the block's sum in shared memory, then one atomic add
// per coupling and block into dJ (N x N, symmetric: both J_ij and J_ji get the value of
// the one parameter).
template <int M>
__global__ void __launch_bounds__(128)
    xy_adjoint_kernel(const __grid_constant__ XYSys S, int64_t count, const double *theta,
                      const double *g_energy, const double *g_theta, double *dJ) {
    constexpr int N = M + 1;
    __shared__ double acc[N * N];
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) {
        const double *J = S.Jd;
        double c[N], s[N], lam[N];
#pragma unroll 1
        for (int k = 0; k < M; k++) sincos(theta[e * M + k], &s[k], &c[k]);
        c[M] = 1.0;
        s[M] = 0.0;
#pragma unroll 1
        for (int k = 0; k < N; k++) lam[k] = 0.0;
        bool ok = true;
        if (g_theta) {
            // H lambda = g by Gaussian elimination with partial pivoting; cos(a - b) =
            // c_a c_b + s_a s_b
            double H[M * M], b[M];
#pragma unroll 1
            for (int k = 0; k < M; k++) {
                double d = 0.0;
#pragma unroll 1
                for (int j = 0; j < N; j++)
                    if (j != k) d += J[k * NPHC_JSTRIDE + j] * (c[k] * c[j] + s[k] * s[j]);
#pragma unroll 1
                for (int l = 0; l < M; l++)
                    H[k * M + l] = (k == l) ? d : -J[k * NPHC_JSTRIDE + l] * (c[k] * c[l] + s[k] * s[l]);
                b[k] = g_theta[e * M + k];
            }
#pragma unroll 1
            for (int k = 0; k < M; k++) {
                int p = k;
#pragma unroll 1
                for (int i = k + 1; i < M; i++)
                    if (fabs(H[i * M + k]) > fabs(H[p * M + k])) p = i;
                if (H[p * M + k] == 0.0) {
                    ok = false;
                    break;
                }
                if (p != k) {
#pragma unroll 1
                    for (int l = 0; l < M; l++) {
                        const double tmp = H[k * M + l];
                        H[k * M + l] = H[p * M + l];
                        H[p * M + l] = tmp;
                    }
                    const double tb = b[k];
                    b[k] = b[p];
                    b[p] = tb;
                }
                const double ip = 1.0 / H[k * M + k];
#pragma unroll 1
                for (int i = k + 1; i < M; i++) {
                    const double f = H[i * M + k] * ip;
#pragma unroll 1
                    for (int l = k + 1; l < M; l++) H[i * M + l] -= f * H[k * M + l];
                    b[i] -= f * b[k];
                }
            }
            if (ok) {
#pragma unroll 1
                for (int k = M - 1; k >= 0; k--) {
                    double v = b[k];
#pragma unroll 1
                    for (int l = k + 1; l < M; l++) v -= H[k * M + l] * lam[l];
                    lam[k] = v / H[k * M + k];
                }
            }
        }
        if (ok) {
            const double gv = g_energy ? g_energy[e] : 0.0;
#pragma unroll 1
            for (int i = 0; i < N; i++)
#pragma unroll 1
                for (int j = i + 1; j < N; j++) {
                    const double cd = c[i] * c[j] + s[i] * s[j];   // cos(theta_i - theta_j)
                    const double sd = s[i] * c[j] - c[i] * s[j];   // sin(theta_i - theta_j)
                    const double v = gv * (1.0 - cd) - (lam[i] - lam[j]) * sd;
                    atomicAdd(&acc[i * N + j], v);
                    atomicAdd(&acc[j * N + i], v);
                }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N * N; i += blockDim.x)
        if (acc[i] != 0.0) atomicAdd(&dJ[i], acc[i]);
}

